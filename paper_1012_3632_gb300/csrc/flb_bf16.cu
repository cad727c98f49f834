// flb_bf16.cu -- kernel instantiation: compute type float, storage type __nv_bfloat16.
#include "flb_prec.cuh"

namespace flb {
const PrecOps& ops_bf16() { return Prec<float, __nv_bfloat16>::ops(); }
}  // namespace flb
