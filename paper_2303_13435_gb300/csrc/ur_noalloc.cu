// ur_fft_intensity_noalloc: the forward transform + binning without a
// caller-supplied workspace.
//
// Who needs this: code that must not allocate device memory when it runs --
// for example a real-time or embedded host loop with a fixed memory budget
// decided at start-up, a plugin whose host application owns every device
// allocation, or a caller that cannot link against or call the CUDA
// allocator at all.  Such a caller still creates its ur_plan during set-up
// (plan creation allocates the plan's small tables), and afterwards can run
// the transform with only its own input and output buffers.
//
// How: the plane-transform intermediate lives in one file-scope device array
// of UR_NOALLOC_SCRATCH_BYTES.  Every GPU that loads this library reserves
// that much device memory for the whole life of the process.  Host code
// cannot use the array's name as a device address (in host code it names a
// host-side stand-in), so the device address is fetched once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; make that first call before any stream capture.  All calls
// share the one array: two calls whose work overlaps on the GPU (for example
// on two streams) overwrite each other's intermediate and give wrong results.
// The array keeps whatever the last call left in it; nothing in it needs to
// start at zero, because the plane pass writes every element of the
// intermediate before the column pass reads it (the bins are cleared in the
// caller's output buffer by the column pass, as in ur_fft_intensity).
#include <mutex>

#include "ur_forward.cuh"

#define UR_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_ur_noalloc_scratch[UR_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[UR_NOALLOC_MAX_DEVICES];

static ur_status noalloc_scratch(const ur_plan* p, void** out) {
  int dev = 0;
  UR_CUDA_CHECK(cudaGetDevice(&dev));
  UR_REQUIRE(dev >= 0 && dev < UR_NOALLOC_MAX_DEVICES, "ur_fft_intensity_noalloc: device %d out of range", dev);
  // the plan's tables live on the device it was created on; the scratch array used must be
  // that device's too
  UR_REQUIRE(dev == p->device, "ur_fft_intensity_noalloc: current device %d is not the plan's device %d", dev,
             p->device);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_ur_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      ur_set_error("ur_fft_intensity_noalloc: cudaGetSymbolAddress of the scratch array failed on device %d: %s", dev,
                   cudaGetErrorString(e));
      return UR_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return UR_OK;
}

extern "C" size_t ur_noalloc_scratch_bytes(void) { return (size_t)UR_NOALLOC_SCRATCH_BYTES; }

extern "C" ur_status ur_fft_intensity_noalloc(const ur_plan* p, const void* ed, double* bins, void* stream) {
  UR_REQUIRE(p && ed && bins, "ur_fft_intensity_noalloc: null argument");
  const size_t need = ur_workspace_size(p, UR_WS_FORWARD);
  UR_REQUIRE(need <= (size_t)UR_NOALLOC_SCRATCH_BYTES,
             "ur_fft_intensity_noalloc: this plan needs %zu bytes of intermediate (nz * N * (N/2+1) * 8); the built-in "
             "scratch holds %zu bytes -- use ur_fft_intensity with a workspace",
             need, (size_t)UR_NOALLOC_SCRATCH_BYTES);
  UR_REQUIRE(((uintptr_t)ed % 8) == 0, "ur_fft_intensity_noalloc: ed must be 8-byte aligned");
  UR_TRY(ur_fault_point("fft_intensity"));
  void* scratch = nullptr;
  UR_TRY(noalloc_scratch(p, &scratch));
  cudaStream_t s = (cudaStream_t)stream;
  float2* X = (float2*)scratch;
  UR_TRY(ur_plane_pass(p, ed, p->nz, X, s));
  UR_TRY(ur_column_pass(p, X, bins, nullptr, s));
  return UR_OK;
}
