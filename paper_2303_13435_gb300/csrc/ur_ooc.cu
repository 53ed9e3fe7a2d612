// Out-of-core forward: the density lives in pinned host memory and is
// streamed to the device slab by slab.  The paper works slice by slice to
// bound memory (Sec. 2.4, intermediates on disk); here slabs of planes go
// host -> HBM over the host link while the plane pass of the previous slab
// runs, and the plane-pass intermediate (only the nz planes that may hold
// density) stays in HBM for the column pass.
//
// Pipeline (two device slab buffers b = i mod 2, one copy stream):
//   copy stream:    wait comp_done[b] (slab i-2 read b) -> H2D slab i -> record copy_done[b]
//   caller stream:  wait copy_done[b] -> plane pass of slab i -> record comp_done[b]
// then the column pass (+ |F|^2 + bins) on the caller stream.  All waits are
// stream/event dependencies: no thread spins on the device.
#include "ur_forward.cuh"

extern "C" ur_status ur_plan_set_slab_planes(ur_plan* p, int32_t planes) {
  UR_REQUIRE(p && planes >= 1, "ur_plan_set_slab_planes: bad argument");
  const size_t ed_plane = (size_t)p->n * p->n * (p->ed_dtype == UR_F16 ? 2 : 4);
  p->slab_planes = planes > p->nz ? p->nz : planes;
  p->ws_slab = (size_t)p->slab_planes * ed_plane;
  return UR_OK;
}

extern "C" ur_status ur_plan_set_chunk_planes(ur_plan* p, int32_t planes) {
  UR_REQUIRE(p && planes >= 1, "ur_plan_set_chunk_planes: bad argument");
  if (!p->fast) return UR_OK;
  const size_t plane_bytes = (size_t)p->n * p->H * sizeof(float2);
  p->chunk_planes = planes > p->n ? p->n : planes;
  // whole-grid passes transform Y in place; chunks need their own buffer
  p->ws_chunk = p->chunk_planes < p->n ? (size_t)p->chunk_planes * plane_bytes : 0;
  return UR_OK;
}

extern "C" int32_t ur_plan_chunk_planes(const ur_plan* p) { return (p && p->fast) ? p->chunk_planes : 0; }

ur_status ur_fft_intensity_host(const ur_plan* p, const void* ed_host, double* bins, float2* F_out, void* ws,
                                size_t ws_bytes, cudaStream_t s) {
  const size_t need = ur_workspace_size(p, UR_WS_FORWARD | UR_WS_HOST_SLABS);
  UR_REQUIRE(ws_bytes >= need, "ur_fft_intensity (host ED): workspace %zu < %zu bytes", ws_bytes, need);
  UR_REQUIRE(((uintptr_t)ws % 256) == 0, "ur_fft_intensity (host ED): misaligned ws");
  {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, ed_host);
    UR_REQUIRE(e == cudaSuccess && at.type == cudaMemoryTypeHost,
               "ur_fft_intensity (host ED): ed must be page-locked host memory (cudaHostAlloc or registered)");
  }
  UR_TRY(ur_fault_point("fft_intensity"));
  const int n = p->n, H = p->H;
  const size_t esz = p->ed_dtype == UR_F16 ? 2 : 4;
  const size_t plane_bytes = (size_t)n * n * esz;
  const int S = p->slab_planes;
  float2* X = (float2*)ws;
  char* slab[2];
  slab[0] = (char*)ws + ur_align_up(p->ws_inter, 256);
  slab[1] = slab[0] + ur_align_up(p->ws_slab, 256);

  cudaStream_t cs = nullptr;
  cudaEvent_t copy_done[2] = {nullptr, nullptr}, comp_done[2] = {nullptr, nullptr};
  ur_status st = UR_OK;
  auto fail = [&](ur_status code) {
    st = code;
    return code;
  };
  do {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      ur_set_error("ur_fft_intensity (host ED): cannot create the copy stream");
      fail(UR_ERR_CUDA);
      break;
    }
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b)
      ok = cudaEventCreateWithFlags(&copy_done[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&comp_done[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      ur_set_error("ur_fft_intensity (host ED): cannot create events");
      fail(UR_ERR_CUDA);
      break;
    }
    // the copy stream starts after everything already queued on the caller stream
    cudaEvent_t start;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) {
      ur_set_error("ur_fft_intensity (host ED): cannot create events");
      fail(UR_ERR_CUDA);
      break;
    }
    cudaEventRecord(start, s);
    cudaStreamWaitEvent(cs, start, 0);
    cudaEventDestroy(start);
    const int nslabs = (p->nz + S - 1) / S;
    for (int i = 0; i < nslabs && st == UR_OK; ++i) {
      const int b = i & 1;
      const int p0 = i * S;
      const int np = (p0 + S <= p->nz) ? S : p->nz - p0;
      if (ur_fault_point("host_slab") != UR_OK) {
        fail(UR_ERR_FAULT_INJECTED);
        break;
      }
      if (i >= 2) cudaStreamWaitEvent(cs, comp_done[b], 0);
      ur_timing_begin("h2d_slab", cs);
      const cudaError_t ce = cudaMemcpyAsync(slab[b], (const char*)ed_host + (size_t)p0 * plane_bytes,
                                             (size_t)np * plane_bytes, cudaMemcpyHostToDevice, cs);
      ur_timing_end(cs);
      if (ce != cudaSuccess) {
        ur_set_error("ur_fft_intensity (host ED): slab copy failed: %s", cudaGetErrorString(ce));
        fail(UR_ERR_CUDA);
        break;
      }
      cudaEventRecord(copy_done[b], cs);
      cudaStreamWaitEvent(s, copy_done[b], 0);
      const ur_status ps = ur_plane_pass(p, slab[b], np, X + (size_t)p0 * n * H, s);
      if (ps != UR_OK) {
        fail(ps);
        break;
      }
      cudaEventRecord(comp_done[b], s);
    }
    if (st == UR_OK) st = ur_column_pass(p, X, bins, F_out, s);
  } while (0);
  // make sure the caller stream does not run ahead of copies still queued on the copy stream
  if (cs) {
    cudaEvent_t end;
    if (cudaEventCreateWithFlags(&end, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(end, cs);
      cudaStreamWaitEvent(s, end, 0);
      cudaEventDestroy(end);
    }
    cudaStreamDestroy(cs);
  }
  for (int b = 0; b < 2; ++b) {
    if (copy_done[b]) cudaEventDestroy(copy_done[b]);
    if (comp_done[b]) cudaEventDestroy(comp_done[b]);
  }
  return st;
}
