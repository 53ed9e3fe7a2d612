// Column pass along z (Sec. 2.4 Eq. 2, outer sum) for grid edges N = 256 and
// 512, fused with |F|^2 and the Sec. 2.5 Q binning: the TMA-staged engine a
// plan selects with ur_plan_set_tma_zpass (the default is the compile-time
// kernel of ur_fast.cu, measured faster at 512^3: 268 against 311 us).
//
// Work unit: a tile of 16 consecutive spectrum columns c = ky_index (N/2+1) + kx
// (the intermediate X[p][ky][kx] seen as rows of N (N/2+1) columns, one row per
// plane holding density).  One thread issues a TMA load of the tile's nz planes
// into shared memory (128-byte swizzle) while the block works on the previous
// tile (two stages, mbarrier completion, bounded waits).  The kernel is
// persistent: one block per SM walks a list of tiles; tiles whose columns all
// lie beyond the last bin are not in the list.
//
// Transform (four-step, N = A * 16): 16 threads per column, two columns per
// warp.  Thread t loads x[16 n1 + t] (n1 < A; planes outside the density slab
// are zero), runs an A-point DFT in registers, multiplies by W_N^(t k1), and
// writes to the warp's exchange buffer; after a warp barrier it reads, for
// k1 in {t, t + 16, ...}, the 16 values Y'[k1][0..15] and runs 16-point DFTs.
// It then holds the spectrum at kz = t + 16 q.  One exchange per transform,
// warp-local barriers only.  The exchange layout swizzles row r to
// r ^ ((r >> 4) & 7) so that both its writes and its reads are free of bank
// conflicts; the natural-order layout used afterwards is unswizzled.
//
// Binning: the spectrum is written in natural order and each thread walks a
// chunk of CH consecutive |kz| = m (with kz = m and N - m), bins only moving
// forward as k^2 = kx^2 + ky^2 + m^2 grows.  A run of equal bins is summed in
// FP32 relative to a per-bin shift K (the first value the block saw in that
// bin): sum (I - K) and sum (I - K)^2.  Runs go into per-block shared
// accumulators (count, shifted sum, shifted sum of squares); at the end each
// block adds, per bin, n mu, n mu^2 and its within-block M2 to FP64 global sums,
// so that the standard error comes from a Chan-style merge of (n, mean, M2)
// and not from the difference of two large sums.
#include <math.h>
#include <mutex>
#include <string.h>

#include <cudaTypedefs.h>

#include "ur_fast.cuh"
#include "ur_tma.cuh"

__device__ int g_ur_deverr = 0;

namespace {

constexpr int ZC_WARPS = 8;
constexpr int ZC_THREADS = 32 * ZC_WARPS;
constexpr int ZC_TILE = 16;  // columns per tile (128 bytes per plane row)
constexpr int ZC_STAGES = 1;  // one tile in flight per block; two blocks per SM
constexpr uint32_t ZC_NAN_BITS = 0x7fc00000u;

struct ZArgs {
  int nz, z0;            // planes of X and the absolute plane of X's first plane
  int box_rows, nbox;    // TMA rows per box (a multiple of 8) and boxes per tile
  int stage_bytes;       // bytes of one stage buffer (a multiple of 1024)
  const int32_t* tiles;  // tile list (first column / 16) or NULL (tile i = i)
  int ntiles;
  const float2* ztw;     // [A][16]: W_N^(t k1) at [k1][t]
  const int32_t* thr;
  const int16_t* lut;    // k^2 -> bin
  int nbins;
  float iscale;          // I' = |F~|^2 * iscale
  const float* vs;       // voxel-sinc factors sinc^2(pi m / N), m <= N/2, or NULL
  double* bins;          // [UR_BIN_FIELDS][nbins], zeroed by the caller; during the pass fields
                         // 1 and 2 hold the shifted sums, field 5 the shifts (ur_bin_shift)
                         // and field 4 slot 0 counts the blocks that are done
  const double* geo;     // plan: per-bin count and sum |Q|
  double inv_n3;
  float2* fout;          // optional F half spectrum [kz][ky][kx]
  float fscale;
};

__host__ __device__ constexpr size_t zc_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

// shared-memory carve-up (the host computes the same sizes)
struct ZLayout {
  size_t stage, xchg, ztw, thr, acc, vs, bars, total;
};
__host__ __device__ inline ZLayout zc_layout(int N, int stage_bytes, int nb) {
  ZLayout L;
  size_t o = 0;
  L.stage = o;
  o += (size_t)ZC_STAGES * stage_bytes;
  L.xchg = o;
  o += (size_t)ZC_WARPS * N * 16;
  L.ztw = o;
  o += (size_t)N * 8;
  L.thr = o;
  o += zc_align((size_t)(nb + 1) * 4, 16);
  L.acc = o;
  o += zc_align((size_t)nb * 12, 16);
  L.vs = o;
  o += zc_align((size_t)(N / 2 + 1) * 4, 16);
  L.bars = o;
  o += (size_t)ZC_STAGES * 8;
  L.total = o + 1024;  // room to align the base to 1024 bytes
  return L;
}

__device__ __forceinline__ void zc_issue(unsigned char* stage, const CUtensorMap* tm, const ZArgs& a, int i,
                                         uint64_t* bar) {
  const int T = a.tiles ? __ldg(a.tiles + i) : i;
  ur_mbar_arrive_expect_tx(bar, (uint32_t)(a.nbox * a.box_rows * 128));
  for (int k = 0; k < a.nbox; ++k) ur_tma_load_2d(stage + (size_t)k * a.box_rows * 128, tm, T * ZC_TILE, k * a.box_rows, bar);
}

template <int N>
__global__ void __launch_bounds__(ZC_THREADS, 2) k_zcol(const __grid_constant__ CUtensorMap tm, ZArgs a) {
  constexpr int M = N / 2, H = M + 1, A = N / 16, NA = A / 16, CH = (H + 15) / 16;
  static_assert(A == 16 || A == 32, "N = 256 or 512");
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = smraw + ((1024u - (ur_smem_u32(smraw) & 1023u)) & 1023u);
  const int nb = a.nbins;
  const ZLayout L = zc_layout(N, a.stage_bytes, nb);
  unsigned char* stage0 = sm + L.stage;
  float2* xchg = reinterpret_cast<float2*>(sm + L.xchg);
  float2* ztw_s = reinterpret_cast<float2*>(sm + L.ztw);
  int32_t* thr_s = reinterpret_cast<int32_t*>(sm + L.thr);
  float* Kb = reinterpret_cast<float*>(sm + L.acc);  // the block's cache of the bin shifts, shifted sums
  float* Sds = Kb + nb;
  float* Qds = Sds + nb;
  float* vs_s = reinterpret_cast<float*>(sm + L.vs);    // voxel-sinc factors (when a.vs)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, t = lane & 15, cw = lane >> 4;
  const int jcol = 2 * warp + cw;
  for (int i = tid; i < A * 16; i += ZC_THREADS) ztw_s[i] = __ldg(a.ztw + i);
  for (int i = tid; i <= nb; i += ZC_THREADS) thr_s[i] = __ldg(a.thr + i);
  if (a.vs)
    for (int i = tid; i <= M; i += ZC_THREADS) vs_s[i] = __ldg(a.vs + i);
  for (int i = tid; i < nb; i += ZC_THREADS) {
    Kb[i] = __int_as_float((int)ZC_NAN_BITS);
    Sds[i] = 0.f;
    Qds[i] = 0.f;
  }
  unsigned long long* gK = ur_shift_slots(a.bins, nb);
  if (tid == 0) {
    for (int s = 0; s < ZC_STAGES; ++s) ur_mbar_init(bars + s, 1);
    ur_fence_barrier_init();
  }
  __syncthreads();
  const int G = gridDim.x;
  if (tid == 0)
    for (int s = 0; s < ZC_STAGES; ++s) {
      const int i = blockIdx.x + s * G;
      if (i < a.ntiles) zc_issue(stage0 + (size_t)s * a.stage_bytes, &tm, a, i, bars + s);
    }

  float2* xw = xchg + (size_t)warp * N * 2;  // this warp's exchange rows: (row, column cw) at row * 2 + cw
  // exchange-write offsets: row 16 k1 + t lives at 16 k1 + (t ^ (k1 & 7))
  int xo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) xo[j] = ((t ^ j) << 1) + cw;
  const int rsw = t & 7;  // exchange-read swizzle of this thread's rows

  int it = 0;
  for (int i = blockIdx.x; i < a.ntiles; i += G, ++it) {
    const int s = it % ZC_STAGES;
    const uint32_t par = (uint32_t)(it / ZC_STAGES) & 1u;
    const bool ok = ur_mbar_wait_bounded(bars + s, par, &g_ur_deverr);
    if (__syncthreads_or(!ok)) {
      // give up: wait (bounded) for the copies still in flight into this block's buffers
      for (int k = 0; k < ZC_STAGES; ++k) {
        const int j = i + k * G;
        if (j < a.ntiles) ur_mbar_wait_bounded(bars + (it + k) % ZC_STAGES, (uint32_t)((it + k) / ZC_STAGES) & 1u, &g_ur_deverr);
      }
      return;
    }
    const int T = a.tiles ? __ldg(a.tiles + i) : i;
    const int col = T * ZC_TILE + jcol;
    const int kyi = col / H, kx = col - kyi * H, ky = kyi < M ? kyi : kyi - N;
    const int c2 = kx * kx + ky * ky;
    // first bin of this thread's chunk of |kz| (issued early; used after the transform)
    const int m0 = CH * t;
    int b0 = nb;
    {
      const int s0 = c2 + m0 * m0;
      if (m0 <= M && s0 < thr_s[nb]) b0 = s0 < thr_s[0] ? -1 : (int)__ldg(a.lut + s0);
    }
    // this column's planes from the stage: row r = z - z0 of the tile, 128-byte swizzle
    float2 v[A];
    {
      const unsigned char* tb = stage0 + (size_t)s * a.stage_bytes;
      const int r0 = t - a.z0;
      const int sw = ((((jcol >> 1) ^ (r0 & 7)) << 4) | ((jcol & 1) << 3));
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) {
        const int r = r0 + 16 * n1;
        v[n1] = (r >= 0 && r < a.nz) ? *reinterpret_cast<const float2*>(tb + (ptrdiff_t)r * 128 + sw)
                                     : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();  // every warp has its columns: the stage may be refilled
    if (tid == 0) {
      const int nx = i + ZC_STAGES * G;
      if (nx < a.ntiles) {
        ur_fence_proxy_async();
        zc_issue(stage0 + (size_t)s * a.stage_bytes, &tm, a, nx, bars + s);
      }
    }
    // ---- forward transform along z ----
    dft<A, false>(v);
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) v[k1] = cmul(v[k1], ztw_s[k1 * 16 + t]);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) xw[32 * k1 + xo[k1 & 7]] = v[k1];
    __syncwarp();
#pragma unroll
    for (int a2 = 0; a2 < NA; ++a2) {
      float2 u[16];
      const int rb = 32 * (t + 16 * a2) + cw;
#pragma unroll
      for (int n2 = 0; n2 < 16; ++n2) u[n2] = xw[rb + ((n2 ^ rsw) << 1)];
      dft<16, false>(u);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) v[a2 + NA * k2] = u[k2];
    }
    __syncwarp();
    // natural order: kz = t + 16 q
#pragma unroll
    for (int q = 0; q < A; ++q) xw[2 * (t + 16 * q) + cw] = v[q];
    if (a.fout) {
#pragma unroll
      for (int q = 0; q < A; ++q) a.fout[(long long)(t + 16 * q) * N * H + col] = cscale(v[q], a.fscale);
    }
    __syncwarp();
    {
      // ---- |F|^2 and Q binning over the chunk m in [m0, m0 + CH) ----
      // Control flow is warp-uniform (votes): the lanes of a warp walk different chunks, and
      // per-lane branches would split the warp for the rest of the walk.
      const float w = (kx == 0 || kx == M) ? 1.f : 2.f;
      const float csc = a.vs ? a.iscale * (vs_s[kx] * vs_s[ky < 0 ? -ky : ky]) : a.iscale;
      int b = b0;
      int tnext = b < nb ? thr_s[b + 1] : 0x7fffffff;
      int s2 = c2 + m0 * m0;
      float sd = 0.f, sd2 = 0.f;
      int cnt = 0;
      // shift of the first run (ur_bin_shift: the first value any block meets in the bin)
      float K = 0.f;
      if (b >= 0 && b < nb) {
        const float2 f0 = xw[2 * m0 + cw];
        const float sc0 = a.vs ? csc * vs_s[m0] : csc;
        K = ur_bin_shift(Kb, gK, b, (f0.x * f0.x + f0.y * f0.y) * sc0);
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int m = m0 + u;
        const float2 f1 = xw[2 * m + cw];
        const float2 f2 = xw[2 * (N - m) + cw];
        const float sc = a.vs ? csc * vs_s[m <= M ? m : M] : csc;
        const float i1 = (f1.x * f1.x + f1.y * f1.y) * sc;
        const float i2 = (f2.x * f2.x + f2.y * f2.y) * sc;
        // a bin change somewhere in the warp: flush, advance and take the new shift (uniform branch)
        bool chg = m <= M && b < nb && s2 >= tnext;
        if (__any_sync(0xffffffffu, chg)) {
          if (chg && cnt > 0) {
            atomicAdd(Sds + b, w * sd);
            atomicAdd(Qds + b, w * sd2);
          }
          const bool moved = chg;
          while (__any_sync(0xffffffffu, chg)) {
            if (chg) {
              ++b;
              tnext = b < nb ? thr_s[b + 1] : 0x7fffffff;
              chg = s2 >= tnext;
            }
          }
          if (moved) {
            sd = sd2 = 0.f;
            cnt = 0;
            if (b < nb) K = ur_bin_shift(Kb, gK, b, i1);
          }
        }
        const bool in = m <= M && b >= 0 && b < nb;
        const float d1 = i1 - K, d2 = i2 - K;
        if (in) {
          sd += d1;
          sd2 = fmaf(d1, d1, sd2);
          ++cnt;
          if (m != 0 && m != M) {
            sd += d2;
            sd2 = fmaf(d2, d2, sd2);
            ++cnt;
          }
        }
        s2 += 2 * m + 1;
      }
      if (cnt > 0 && b >= 0 && b < nb) {
        atomicAdd(Sds + b, w * sd);
        atomicAdd(Qds + b, w * sd2);
      }
    }
    __syncwarp();
  }
  {
    __syncthreads();
    for (int j = tid; j < nb; j += ZC_THREADS) {
      if (Sds[j] != 0.f) atomicAdd(a.bins + UR_BIN_SUM_I * nb + j, (double)Sds[j]);
      if (Qds[j] != 0.f) atomicAdd(a.bins + UR_BIN_SUM_I2 * nb + j, (double)Qds[j]);
    }
    // the last block to finish turns the shifted sums into the bin statistics
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (tid == 0)
      s_last = atomicAdd(reinterpret_cast<unsigned long long*>(a.bins + UR_BIN_MEAN * nb), 1ull) ==
               (unsigned long long)(gridDim.x - 1);
    __syncthreads();
    if (s_last) {
      __threadfence();
      for (int j = tid; j < nb; j += ZC_THREADS) {
        // the sums and shifts of the other blocks are in L2
        a.bins[UR_BIN_SUM_I * nb + j] = __ldcg(a.bins + UR_BIN_SUM_I * nb + j);
        a.bins[UR_BIN_SUM_I2 * nb + j] = __ldcg(a.bins + UR_BIN_SUM_I2 * nb + j);
        a.bins[UR_BIN_SEM * nb + j] = __ldcg(a.bins + UR_BIN_SEM * nb + j);
      }
      __syncthreads();
      // (slot 0 of the mean field held the block counter; finalize overwrites it)
      for (int j = tid; j < nb; j += ZC_THREADS) ur_finalize_shifted(a.bins, a.geo, nb, a.inv_n3, j);
    }
  }
}

// driver entry point of the tensor-map encoder, fetched once
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

}  // namespace

ur_status ur_tmap_2d_u64(CUtensorMap* out, const void* base, uint64_t d0, uint64_t d1, uint64_t stride1, uint32_t b0,
                         uint32_t b1, bool swz128) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (g_encode_err == cudaSuccess && q == cudaDriverEntryPointSuccess) g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) {
    ur_set_error("cuTensorMapEncodeTiled is not available: %s", cudaGetErrorString(g_encode_err));
    return UR_ERR_UNSUPPORTED;
  }
  UR_REQUIRE(((uintptr_t)base % 16) == 0 && stride1 % 16 == 0 && b0 * 8 % 16 == 0 && b0 <= 256 && b1 <= 256,
             "tensor map: misaligned base or stride, or box too large");
  const cuuint64_t dims[2] = {d0, d1};
  const cuuint64_t strides[1] = {stride1};
  const cuuint32_t box[2] = {b0, b1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, swz128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    ur_set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return UR_ERR_CUDA;
  }
  return UR_OK;
}

// Test hook: a block waits on an mbarrier that nothing completes, with a short limit
// (about 2^24 cycles); the wait gives up, sets the device error word and the kernel
// returns, so the next ur_sync_status reports UR_ERR_TIMEOUT.  No device fault.
__global__ void k_selftest_wait_timeout() {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ur_mbar_init(&bar, 1);
    ur_fence_barrier_init();
  }
  __syncthreads();
  ur_mbar_wait_bounded(&bar, 0, &g_ur_deverr, 1ll << 24);
}

extern "C" ur_status ur_selftest_wait_timeout(void* stream) {
  k_selftest_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>();
  UR_LAUNCH_CHECK("k_selftest_wait_timeout");
  return UR_OK;
}

ur_status ur_deverr_take(void) {
  int h = 0;
  UR_CUDA_CHECK(cudaMemcpyFromSymbol(&h, g_ur_deverr, sizeof h));
  if (h) {
    const int z = 0;
    UR_CUDA_CHECK(cudaMemcpyToSymbol(g_ur_deverr, &z, sizeof z));
    ur_set_error("a device-side wait gave up (error word %d)", h);
    return UR_ERR_TIMEOUT;
  }
  return UR_OK;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
bool ur_zcol_supported(const ur_plan* p) { return p->zc_tw != nullptr; }

extern "C" ur_status ur_plan_set_tma_zpass(ur_plan* p, int32_t on) {
  UR_REQUIRE(p, "ur_plan_set_tma_zpass: null plan");
  if (on && !ur_zcol_supported(p)) {
    ur_set_error("ur_plan_set_tma_zpass: the TMA z pass is built for N = 256 and 512 with at most 1024 bins");
    return UR_ERR_UNSUPPORTED;
  }
  p->zc_enabled = on ? 1 : 0;
  return UR_OK;
}

extern "C" int32_t ur_plan_tma_zpass(const ur_plan* p) { return (p && p->zc_enabled) ? 1 : 0; }

ur_status ur_zcol_prepare(ur_plan* p) {
  p->zc_tw = nullptr;
  p->zc_tiles = nullptr;
  p->zc_ntiles = 0;
  const int n = p->n;
  if (!(n == 256 || n == 512) || p->nbins > 1024) return UR_OK;
  const int A = n / 16, H = n / 2 + 1, M = n / 2;
  float2* tw = (float2*)malloc(sizeof(float2) * A * 16);
  for (int k1 = 0; k1 < A; ++k1)
    for (int t = 0; t < 16; ++t) {
      const double ang = 2.0 * M_PI * (double)(t * k1) / (double)n;
      tw[k1 * 16 + t] = make_float2((float)cos(ang), (float)(-sin(ang)));
    }
  // tiles with at least one column below the closing threshold
  const long long ntile_all = (long long)n * H / ZC_TILE;
  int32_t* tl = (int32_t*)malloc(sizeof(int32_t) * ntile_all);
  int cnt = 0;
  const int64_t tb = p->thr_host[p->nbins];
  for (long long T = 0; T < ntile_all; ++T) {
    bool keep = false;
    for (int j = 0; j < ZC_TILE && !keep; ++j) {
      const long long c = T * ZC_TILE + j;
      const int kyi = (int)(c / H), kx = (int)(c % H), ky = kyi < M ? kyi : kyi - n;
      keep = (int64_t)kx * kx + (int64_t)ky * ky < tb;
    }
    if (keep) tl[cnt++] = (int32_t)T;
  }
  cudaError_t e1 = cudaMalloc(&p->zc_tw, sizeof(float2) * A * 16);
  cudaError_t e2 = cudaMalloc(&p->zc_tiles, sizeof(int32_t) * (cnt > 0 ? cnt : 1));
  if (e1 == cudaSuccess) e1 = cudaMemcpy(p->zc_tw, tw, sizeof(float2) * A * 16, cudaMemcpyHostToDevice);
  if (e2 == cudaSuccess && cnt > 0) e2 = cudaMemcpy(p->zc_tiles, tl, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice);
  free(tw);
  free(tl);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    ur_set_error("z-column tables: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return UR_ERR_OOM;
  }
  p->zc_ntiles = cnt;
  return UR_OK;
}

template <int N>
static ur_status zcol_launch(const ur_plan* p, const CUtensorMap& tm, ZArgs a, cudaStream_t s) {
  const ZLayout L = zc_layout(N, a.stage_bytes, a.nbins);
  UR_REQUIRE(L.total <= 227 * 1024, "z column pass: %zu bytes of shared memory (max 227 KB)", L.total);
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_zcol<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  int per_sm = 0;
  UR_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_zcol<N>, ZC_THREADS, L.total));
  if (per_sm < 1) per_sm = 1;
  int grid = p->num_sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid <= 0) return UR_OK;
  k_zcol<N><<<grid, ZC_THREADS, L.total, s>>>(tm, a);
  UR_LAUNCH_CHECK("k_zcol");
  return UR_OK;
}

static ur_status zcol_common(const ur_plan* p, const float2* X, ZArgs& a, CUtensorMap& tm) {
  const int n = p->n, H = p->H;
  memset(&a, 0, sizeof a);
  a.nz = p->nz;
  a.z0 = p->z0;
  a.nbox = (p->nz + 255) / 256;
  a.box_rows = (int)zc_align((size_t)((p->nz + a.nbox - 1) / a.nbox), 8);
  a.stage_bytes = (int)zc_align((size_t)a.nbox * a.box_rows * 128, 1024);
  a.ztw = p->zc_tw;
  a.thr = p->thr;
  a.lut = p->binlut;
  a.nbins = p->nbins;
  return ur_tmap_2d_u64(&tm, X, (uint64_t)n * H, (uint64_t)p->nz, (uint64_t)n * H * 8, ZC_TILE, (uint32_t)a.box_rows,
                        true);
}

// Forward column pass with binning and optional F: bins (zeroed by the caller) hold the
// finished statistics when the kernel ends (its last block finalizes them).
ur_status ur_zcol_forward(const ur_plan* p, const float2* X, double* bins, float2* F_out, float iscale, float fscale,
                          cudaStream_t s) {
  ZArgs a;
  CUtensorMap tm;
  UR_TRY(zcol_common(p, X, a, tm));
  const int nb = p->nbins;
  a.tiles = F_out ? nullptr : p->zc_tiles;
  a.ntiles = F_out ? (int)((long long)p->n * p->H / ZC_TILE) : p->zc_ntiles;
  a.iscale = iscale;
  a.vs = p->vsinc;
  a.bins = bins;
  a.geo = p->geo;
  a.inv_n3 = 1.0 / ((double)p->n * p->n * p->n);
  a.fout = F_out;
  a.fscale = fscale;
  if (p->n == 512) return zcol_launch<512>(p, tm, a, s);
  return zcol_launch<256>(p, tm, a, s);
}
