// flb_fp32.cu -- kernel instantiation: compute type float, storage type float.
#include "flb_prec.cuh"

namespace flb {
const PrecOps& ops_fp32() { return Prec<float, float>::ops(); }
}  // namespace flb
