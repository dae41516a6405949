// Split-BF16 tensor-core operators (tcgen05 / TMEM).  Placeholder until the
// tensor-core path lands: models built with OAM_PREC_BF16X3 are rejected.
#include "internal.cuh"

namespace oam {
struct TcLayout {};
oam_status tc_build(oam_model *, cudaStream_t) { return OAM_ERR_UNSUPPORTED; }
void tc_free(oam_model *) {}
oam_status forward_tc(const oam_model *, const float *, float *, cudaStream_t) { return OAM_ERR_UNSUPPORTED; }
oam_status adjoint_tc(const oam_model *, const float *, float *, cudaStream_t) { return OAM_ERR_UNSUPPORTED; }
}  // namespace oam
