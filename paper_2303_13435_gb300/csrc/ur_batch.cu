// Batched particles of uneven grid sizes.
#include "ur_forward.cuh"

extern "C" size_t ur_batch_workspace_size(int32_t count, const ur_plan* const* plans, int32_t what) {
  size_t b = 0;
  for (int i = 0; i < count; ++i) b += ur_align_up(ur_workspace_size(plans[i], what), 256);
  return b;
}

extern "C" ur_status ur_batch_forward(int32_t count, const ur_plan* const* plans, const void* const* eds, double* const* bins,
                                      void* ws, size_t ws_bytes, void* stream) {
  (void)count;
  (void)plans;
  (void)eds;
  (void)bins;
  (void)ws;
  (void)ws_bytes;
  (void)stream;
  ur_set_error("ur_batch_forward: not built yet");
  return UR_ERR_UNSUPPORTED;
}
