// flb_fp64.cu -- kernel instantiation: compute type double, storage type double.
#include "flb_prec.cuh"

namespace flb {
const PrecOps& ops_fp64() { return Prec<double, double>::ops(); }
}  // namespace flb
