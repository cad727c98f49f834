// flb_fp32.cu -- kernel instantiation: compute type float, storage type float.
#include "flb_prec.cuh"

namespace flb {
const PrecOps& ops_fp32() { return Prec<float, float>::ops(); }
Coll<float> coll_fp32(const HostModel& m, uint64_t step) { return make_coll<D3Q19, float>(m, step); }
}  // namespace flb
