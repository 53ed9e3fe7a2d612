// Out-of-core forward: the density lives in pinned host memory and is
// streamed to the device slab by slab (Sec. 2.4 works slice by slice to bound
// memory; here the slabs go host -> HBM instead of disk -> RAM).
#include "ur_forward.cuh"

ur_status ur_fft_intensity_host(const ur_plan* p, const void* ed_host, double* bins, float2* F_out, void* ws,
                                size_t ws_bytes, cudaStream_t s) {
  (void)p;
  (void)ed_host;
  (void)bins;
  (void)F_out;
  (void)ws;
  (void)ws_bytes;
  (void)s;
  ur_set_error("ur_fft_intensity: host-resident density not built yet");
  return UR_ERR_UNSUPPORTED;
}
