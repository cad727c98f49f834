// flb_fp64.cu -- kernel instantiation: compute type double, storage type double.
#include "flb_prec.cuh"

namespace flb {
const PrecOps& ops_fp64() { return Prec<double, double>::ops(); }
Coll<double> coll_fp64(const HostModel& m, uint64_t step) { return make_coll<D3Q19, double>(m, step); }
}  // namespace flb
