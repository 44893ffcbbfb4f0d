// Backward pass of the render path (placeholder until the gradient kernels land).
#include "internal.h"

extern "C" hg_status hg_render_backward(hg_state* state, const float* dL_drgb, float* d_means, float* d_log_scales,
                                        float* d_quats, float* d_opacity_logits, float* d_sh, void* stream) {
  (void)state, (void)dL_drgb, (void)d_means, (void)d_log_scales, (void)d_quats, (void)d_opacity_logits,
      (void)d_sh, (void)stream;
  hg_set_error("hg_render_backward: not available in this build");
  return HG_ERR_UNSUPPORTED;
}
