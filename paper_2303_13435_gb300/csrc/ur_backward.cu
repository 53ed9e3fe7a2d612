// Adjoint of the forward map (not in the paper; the chain rule through
// Sec. 2.3-2.5).  For g_j = dL/d(mean I_j) and G_k = g_j / n_j on bin j:
//
//   dL/drho(x) = (2/N^3) Re sum_k G_k F_k e^{+2 pi i k.x/N}
//              = (1/N^3) Re sum_k sigma_j F~_k e^{+2 pi i k.x/N},  sigma_j = 2 g_j / (n_j N^3)
//
// with F~ the unnormalised transform.  The inverse transform runs in the
// reverse order of the forward passes:
//   B1 k_cols<COL_ZADJ>  per (ky, kx) column: F~ along z recomputed from the
//                        forward intermediate (or F read), times sigma(bin),
//                        inverse transform along z, all N planes written
//   B2 k_cols<COL_Y,inv> inverse transform along y of every plane, in place
//   B3 k_rows_grad       inverse real transform along x of every row, then
//                        dL/dm = dL/drho * u(x mod U) written and
//                        dL/du(c) = sum over tiles of dL/drho * m(x) reduced;
//                        a block takes a batch of the grid rows that wrap
//                        onto one cell row (cz, cy), so its partial sums of
//                        dL/du land on one cell row (one global add each).
#include <math.h>
#include <string.h>

#include "ur_fast.cuh"

// sigma_j = 2 g_j / (n_j N^3) (scale of F~), or 2 g_j / n_j when F (= F~/N^3) is read
__global__ void k_sigma(const double* __restrict__ g, const double* __restrict__ fwd_bins, int nb, double n3, int f_given,
                        float* __restrict__ sigma) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const double n = fwd_bins[UR_BIN_COUNT * nb + j];
  double v = 0.0;
  if (n > 0) v = 2.0 * g[j] / n / (f_given ? 1.0 : n3);
  sigma[j] = (float)v;
}

// B3.  Block (cz, cy); rows (z, y) with (z+oz) mod U = cz and (y+oy) mod U = cy.
// Each row: Y[z][y][0..M] (Hermitian half along x) -> Z[k] = E[k] + i O[k],
//   E[k] = X[k] + conj X[M-k],  O[k] = (X[k] - conj X[M-k]) conj(W_N^k),
// then z = IFFT_{M}(Z) gives (g(2m), g(2m+1)) = (Re z[m], Im z[m]).
struct NoStore {
  __device__ __forceinline__ void operator()(int, int, float2) const {}
};

__device__ __forceinline__ void rows_grad_body(const GenGradArgs& g, int bx, int by) {
  const float2* __restrict__ Y = g.Y;
  const int N = g.N, RB = g.RB, nst = g.nst, U = g.U, ox = g.ox, oy = g.oy, oz = g.oz;
  const StageInfo* __restrict__ sched = g.sched;
  const float2* __restrict__ tw = g.tw;
  const float* __restrict__ cell = g.cell;
  const ShapeArgs& sh = g.sh;
  const float* __restrict__ weights = g.weights;
  const float inv_n3 = g.inv_n3;
  float* __restrict__ dl_dmask = g.dl_dmask;
  float* __restrict__ dl_dcell = g.dl_dcell;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int M = N >> 1, H = M + 1;
  float2* buf = reinterpret_cast<float2*>(smraw);
  float* acc = reinterpret_cast<float*>(smraw + ur_align_up_dev((size_t)RB * H * sizeof(float2), 16));
  const int cz = by / U, cy = by - (by / U) * U;
  const int zf = ((cz - oz) % U + U) % U, yf = ((cy - oy) % U + U) % U;
  const int nzr = zf < N ? (N - 1 - zf) / U + 1 : 0;
  const int nyr = yf < N ? (N - 1 - yf) / U + 1 : 0;
  const int nrows = nzr * nyr;
  const int r0 = bx * RB;
  if (r0 >= nrows) return;  // uniform over the block
  for (int i = threadIdx.x; i < U; i += blockDim.x) acc[i] = 0.f;
  const float* crow = cell + ((long long)cz * U + cy) * U;
  const FastDiv dM((uint32_t)M), dH((uint32_t)H), dNy((uint32_t)(nyr > 0 ? nyr : 1)), dU((uint32_t)U);
  __syncthreads();
  {
    const int nb = min(RB, nrows - r0);
    if (nst >= 2) {
      // the first stage packs its inputs straight from the Hermitian half rows (no staging
      // round trip): Z[i] = (X[i] + conj X[M-i]) + i (X[i] - conj X[M-i]) conj(W_N^i), X[M] for i = 0
      auto packed = [&](int t, int i) -> float2 {
        if (t >= nb) return make_float2(0.f, 0.f);
        const int q = r0 + t;
        const int a = (int)dNy.div((uint32_t)q);
        const int b = q - a * nyr;
        const long long z = zf + (long long)U * a, y = yf + (long long)U * b;
        const float2* row = Y + (z * N + y) * H;
        const float2 xa = __ldg(row + i), xb = __ldg(row + (M - i));
        const float2 w = __ldg(tw + i);
        const float2 e = cadd(xa, cconj(xb));
        const float2 d = csub(xa, cconj(xb));
        const float2 o = make_float2(d.x * w.x + d.y * w.y, d.y * w.x - d.x * w.y);  // * conj(W^i)
        return make_float2(e.x - o.y, e.y + o.x);
      };
      fft_lines_io<true, UR_EMAX, true, false, false>(buf, H, RB, sched, nst, tw, packed, NoStore());
    } else {
      for (int f = threadIdx.x; f < RB * H; f += blockDim.x) {
        const int t = (int)dH.div((uint32_t)f);
        const int k = f - t * H;
        float2 v = make_float2(0.f, 0.f);
        if (t < nb) {
          const int q = r0 + t;
          const int a = (int)dNy.div((uint32_t)q);
          const int b = q - a * nyr;
          const long long z = zf + (long long)U * a, y = yf + (long long)U * b;
          v = __ldg(Y + (z * N + y) * H + k);
        }
        buf[f] = v;
      }
      __syncthreads();
      // Hermitian half -> packed complex sequence, in place by (k, M-k) pairs
      const int half = M / 2 + 1;
      const FastDiv dhalf((uint32_t)half);
      for (int f = threadIdx.x; f < RB * half; f += blockDim.x) {
        const int t = (int)dhalf.div((uint32_t)f);
        const int k = f - t * half;
        float2* X = buf + t * H;
        const float2 xa = X[k], xb = X[M - k];
        const float2 wa = __ldg(tw + k);
        // Z[k]
        const float2 ea = cadd(xa, cconj(xb));
        const float2 da = csub(xa, cconj(xb));
        const float2 oa = make_float2(da.x * wa.x + da.y * wa.y, da.y * wa.x - da.x * wa.y);  // * conj(W^k)
        const float2 za = make_float2(ea.x - oa.y, ea.y + oa.x);
        if (k != 0 && 2 * k != M) {
          const float2 wb = __ldg(tw + (M - k));
          const float2 eb = cadd(xb, cconj(xa));
          const float2 db = csub(xb, cconj(xa));
          const float2 ob = make_float2(db.x * wb.x + db.y * wb.y, db.y * wb.x - db.x * wb.y);
          X[M - k] = make_float2(eb.x - ob.y, eb.y + ob.x);
        }
        X[k] = za;
      }
      __syncthreads();
      fft_lines<true, UR_EMAX>(buf, H, RB, sched, nst, tw);
    }
    // epilogue
    for (int f = threadIdx.x; f < RB * M; f += blockDim.x) {
      const int t = (int)dM.div((uint32_t)f);
      const int m = f - t * M;
      if (t >= nb) continue;
      const int q = r0 + t;
      const int a = (int)dNy.div((uint32_t)q);
      const int b = q - a * nyr;
      const int z = zf + U * a, y = yf + U * b;
      const float2 zv = buf[t * H + m];
      const float g0 = zv.x * inv_n3, g1 = zv.y * inv_n3;
      const int x0 = 2 * m;
      const int c0 = (int)dU.mod((uint32_t)(x0 + ox)), c1 = (int)dU.mod((uint32_t)(x0 + 1 + ox));
      const long long vox = ((long long)z * N + y) * N + x0;
      if (dl_dmask) {
        const float u0 = __ldg(crow + c0), u1 = __ldg(crow + c1);
        *reinterpret_cast<float2*>(dl_dmask + vox) = make_float2(g0 * u0, g1 * u1);
      }
      float m0, m1;
      if (sh.kind == UR_SHAPE_WEIGHTS) {
        const float2 wv = __ldg(reinterpret_cast<const float2*>(weights + vox));
        m0 = wv.x;
        m1 = wv.y;
      } else {
        m0 = mask_at(sh, x0, y, z);
        m1 = mask_at(sh, x0 + 1, y, z);
      }
      if (m0 != 0.f) atomicAdd(acc + c0, g0 * m0);
      if (m1 != 0.f) atomicAdd(acc + c1, g1 * m1);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < U; i += blockDim.x)
    if (acc[i] != 0.f) atomicAdd(dl_dcell + ((long long)cz * U + cy) * U + i, acc[i]);
}

__global__ void __launch_bounds__(256, 4) k_rows_grad(GenGradArgs g) { rows_grad_body(g, blockIdx.x, blockIdx.y); }

// Log-I(Q) MSE and its gradient: one thread per bin over blocks of 64 threads
// (the float64 logarithms are the cost, so they are spread over many SMs).
// Every block first counts the valid bins of the whole curve (V, needed by the
// gradient of every bin; a cheap scan), then writes its bins' gradients and
// adds its share of L = sum d^2 / V to *loss (zeroed beforehand).  float64
// throughout.
#define UR_LOSS_THREADS 64
#define UR_LOSS_MAX_BINS 8192
__global__ void __launch_bounds__(UR_LOSS_THREADS) k_log_mse_grad(int nb, const double* __restrict__ bins,
                                                                  const double* __restrict__ target,
                                                                  double* __restrict__ loss, double* __restrict__ g) {
  __shared__ int s_cnt[UR_LOSS_THREADS / 32];
  __shared__ double s_sum[UR_LOSS_THREADS / 32];
  const double* mean = bins + (size_t)UR_BIN_MEAN * nb;
  int cnt = 0;
  for (int j = threadIdx.x; j < nb; j += UR_LOSS_THREADS) {
    const double m = mean[j];
    cnt += (isfinite(m) && m > 0.0) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  int ntot = 0;
  for (int w = 0; w < UR_LOSS_THREADS / 32; ++w) ntot += s_cnt[w];
  const double nv = (double)(ntot > 0 ? ntot : 1);
  const int j = blockIdx.x * UR_LOSS_THREADS + threadIdx.x;
  double d2 = 0.0;
  if (j < nb) {
    const double m = mean[j];
    double gj = 0.0;
    if (isfinite(m) && m > 0.0) {
      const double d = log(m) - log(target[j]);
      d2 = d * d;
      gj = 2.0 * d / (m * nv);
    }
    g[j] = gj;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d2 += __shfl_down_sync(0xffffffffu, d2, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = d2;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    double tot = 0.0;
    for (int w = 0; w < UR_LOSS_THREADS / 32; ++w) tot += s_sum[w];
    if (tot != 0.0) atomicAdd(loss, tot / nv);
  }
}

extern "C" ur_status ur_log_mse_grad(int32_t nbins, const double* bins, const double* target, double* loss,
                                     double* dl_dmean, void* stream) {
  UR_REQUIRE(nbins >= 1 && bins && target && dl_dmean, "ur_log_mse_grad: bad argument");
  UR_REQUIRE(nbins <= UR_LOSS_MAX_BINS, "ur_log_mse_grad: %d bins (at most %d)", nbins, UR_LOSS_MAX_BINS);
  cudaStream_t s = (cudaStream_t)stream;
  ur_timing_begin("loss_grad", s);
  if (loss) UR_CUDA_CHECK(cudaMemsetAsync(loss, 0, sizeof(double), s));
  k_log_mse_grad<<<(nbins + UR_LOSS_THREADS - 1) / UR_LOSS_THREADS, UR_LOSS_THREADS, 0, s>>>(nbins, bins, target, loss,
                                                                                              dl_dmean);
  UR_LAUNCH_CHECK("k_log_mse_grad");
  ur_timing_end(s);
  return UR_OK;
}

extern "C" ur_status ur_backward(const ur_plan* p, const double* dl_dmean, const double* fwd_bins, const void* F,
                                 const float* cell, int32_t ucell, const int32_t* origin, const ur_shape* shape,
                                 const float* weights, float* dl_dcell, float* dl_dmask, void* ws, size_t ws_bytes,
                                 void* stream) {
  UR_REQUIRE(p && dl_dmean && fwd_bins && cell && shape && dl_dcell && ws, "ur_backward: null argument");
  UR_REQUIRE(ucell >= 1, "ur_backward: empty cell");
  UR_REQUIRE(!origin || (origin[0] >= 0 && origin[1] >= 0 && origin[2] >= 0), "ur_backward: origin must be >= 0");
  UR_REQUIRE(ws_bytes >= ur_workspace_size(p, UR_WS_FORWARD | UR_WS_BACKWARD), "ur_backward: workspace %zu < %zu bytes",
             ws_bytes, ur_workspace_size(p, UR_WS_FORWARD | UR_WS_BACKWARD));
  UR_REQUIRE(shape->kind >= UR_SHAPE_SPHERE && shape->kind <= UR_SHAPE_WEIGHTS, "ur_backward: bad shape kind");
  UR_REQUIRE(shape->kind != UR_SHAPE_WEIGHTS || weights, "ur_backward: weights required for UR_SHAPE_WEIGHTS");
  UR_REQUIRE(!dl_dmask || ((uintptr_t)dl_dmask % 8) == 0, "ur_backward: dl_dmask must be 8-byte aligned");
  if (p->vsinc) {
    ur_set_error("ur_backward: the adjoint of the voxel-sinc corrected binning is not built");
    return UR_ERR_UNSUPPORTED;
  }
  UR_TRY(ur_fault_point("backward"));
  cudaStream_t s = (cudaStream_t)stream;
  const int n = p->n, H = p->H, nb = p->nbins;
  const double n3 = (double)n * n * n;
  float2* X = (float2*)ws;
  float2* Y = (float2*)((char*)ws + ur_align_up(p->ws_inter, 256));
  float* sigma = (float*)((char*)Y + ur_align_up(p->ws_inv, 256));

  ur_timing_begin("sigma", s);
  k_sigma<<<(nb + 255) / 256, 256, 0, s>>>(dl_dmean, fwd_bins, nb, n3, F != nullptr, sigma);
  UR_LAUNCH_CHECK("k_sigma");
  ur_timing_end(s);

  // B1
  ColArgs a = ur_col_args(p);
  a.ncols = (long long)n * H;
  a.A = H;
  a.S = (long long)n * H;
  a.Ad = H;
  a.Sd = (long long)n * H;
  a.dst = Y;
  a.sigma = sigma;
  if (F) {
    a.src = (const float2*)F;
    a.nload = n;
    a.zoff = 0;
    a.skip_fwd = 1;
  } else {
    a.src = X;
    a.nload = p->nz;
    a.zoff = p->z0;
    a.skip_fwd = 0;
  }
  const long long tiles = (a.ncols + a.TX - 1) / a.TX;
  // power-of-two path: columns with kx^2 + ky^2 at or beyond the closing threshold get zero
  // scales at every kz; the z pass leaves them unwritten and the y pass reads them as zeros
  const int k2_zero = p->fast ? (int)(p->thr_host[nb] < 0x7fffffff ? p->thr_host[nb] : 0x7fffffff) : 0x7fffffff;
  if (p->fast) a.k2_zero = k2_zero;
  ur_timing_begin("adj_cols_z", s);
  if (p->fast) {
    UR_TRY(ur_fast_cols(n, 3 /* z adjoint */, a, s));
  } else {
    UR_TRY(ur_launch_cols(COL_ZADJ, false, p, a, (int)tiles, p->col_smem, s));
  }
  ur_timing_end(s);

  if (p->fast) {
    // B2 + B3, over all planes with the y-inverse in place, or in plane chunks
    // whose y-inverse goes to a chunk buffer that the row pass of the same chunk
    // reads while it is still in L2.
    UR_REQUIRE(!weights || ((uintptr_t)weights % 8) == 0, "ur_backward: weights must be 8-byte aligned");
    const bool whole = p->chunk_planes >= n;
    float2* C = (float2*)((char*)sigma + ur_align_up(p->ws_sigma, 256));
    GradArgs g;
    memset(&g, 0, sizeof g);
    g.tw = p->tw;
    g.stw = p->stw + p->stw_m_off;
    g.cell = cell;
    g.ucell = ucell;
    if (origin) {  // the row kernel takes the origin reduced modulo the cell edge
      g.ox = origin[0] % ucell;
      g.oy = origin[1] % ucell;
      g.oz = origin[2] % ucell;
    }
    g.sh = ur_shape_args(shape);
    g.weights = shape->kind == UR_SHAPE_WEIGHTS ? weights : nullptr;
    g.inv_n3 = (float)(1.0 / n3);
    g.dl_dmask = dl_dmask;
    g.dl_dcell = dl_dcell;
    UR_CUDA_CHECK(cudaMemsetAsync(dl_dcell, 0, sizeof(float) * (size_t)ucell * ucell * ucell, s));
    for (int p0 = 0; p0 < n; p0 += p->chunk_planes) {
      const int np = (p0 + p->chunk_planes <= n) ? p->chunk_planes : n - p0;
      ColArgs b = ur_col_args(p);
      b.src = Y + (long long)p0 * n * H;
      b.dst = whole ? Y : C;
      b.ncols = (long long)np * H;
      b.A = (long long)n * H;
      b.S = H;
      b.Ad = b.A;
      b.Sd = b.S;
      b.nload = n;
      b.zoff = 0;
      b.nbins = 0;
      b.k2_zero = k2_zero;
      ur_timing_begin("adj_cols_y", s);
      UR_TRY(ur_fast_cols(n, 1 /* y inverse */, b, s));
      ur_timing_end(s);
      g.Y = whole ? Y : C;
      g.ybase_z = p0;
      g.z0 = p0;
      ur_timing_begin("adj_rows_grad", s);
      UR_TRY(ur_fast_rows_grad(n, g, np, s));
      ur_timing_end(s);
    }
    return UR_OK;
  }

  // B2
  ColArgs b = ur_col_args(p);
  b.src = Y;
  b.dst = Y;
  b.ncols = (long long)n * H;
  b.A = (long long)n * H;
  b.S = H;
  b.Ad = b.A;
  b.Sd = b.S;
  b.nload = n;
  b.zoff = 0;
  b.nbins = 0;
  ur_timing_begin("adj_cols_y", s);
  UR_TRY(ur_launch_cols(COL_Y, true, p, b, (int)tiles, p->col_smem, s));
  ur_timing_end(s);

  // B3
  const ShapeArgs sh = ur_shape_args(shape);
  int ox = 0, oy = 0, oz = 0;
  if (origin) {
    ox = origin[0];
    oy = origin[1];
    oz = origin[2];
  }
  const int RB = p->row_rb;
  const size_t smem = ur_align_up((size_t)RB * H * sizeof(float2), 16) + (size_t)ucell * sizeof(float);
  UR_REQUIRE(smem <= 227 * 1024, "ur_backward: cell edge %d too large for the row reduction", ucell);
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_rows_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  UR_REQUIRE((long long)ucell * ucell <= 65535, "ur_backward: cell edge %d too large", ucell);
  const int rows_per_group = ((n + ucell - 1) / ucell) * ((n + ucell - 1) / ucell);
  dim3 ggrid((unsigned)((rows_per_group + RB - 1) / RB), (unsigned)(ucell * ucell));
  UR_CUDA_CHECK(cudaMemsetAsync(dl_dcell, 0, sizeof(float) * (size_t)ucell * ucell * ucell, s));
  ur_timing_begin("adj_rows_grad", s);
  GenGradArgs ga;
  memset(&ga, 0, sizeof ga);
  ga.Y = Y;
  ga.N = n;
  ga.RB = RB;
  ga.nst = p->sched_m.nst;
  ga.sched = p->d_sched + UR_MAX_STAGES;
  ga.tw = p->tw;
  ga.cell = cell;
  ga.U = ucell;
  ga.ox = ox;
  ga.oy = oy;
  ga.oz = oz;
  ga.sh = sh;
  ga.weights = shape->kind == UR_SHAPE_WEIGHTS ? weights : nullptr;
  ga.inv_n3 = (float)(1.0 / n3);
  ga.dl_dmask = dl_dmask;
  ga.dl_dcell = dl_dcell;
  k_rows_grad<<<ggrid, 256, smem, s>>>(ga);
  UR_LAUNCH_CHECK("k_rows_grad");
  ur_timing_end(s);
  return UR_OK;
}

// ---------------------------------------------------------------------------
// Batched adjoint launches
// ---------------------------------------------------------------------------
__global__ void k_batch_sigma(const BatchSigmaItem* __restrict__ items) {
  const BatchSigmaItem& it = items[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= it.nb) return;
  const double n = it.bins[UR_BIN_COUNT * it.nb + j];
  it.sigma[j] = (float)(n > 0 ? 2.0 * it.g[j] / n / it.n3 : 0.0);
}

__global__ void __launch_bounds__(256, 4) k_batch_grad(const BatchGradItem* __restrict__ items,
                                                       const long long* __restrict__ start, int count) {
  int lo = 0, hi = count - 1;
  const long long b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  const BatchGradItem& it = items[lo];
  const long long local = b - __ldg(start + lo);
  const int gx = it.gx;
  rows_grad_body(it.g, (int)(local % gx), (int)(local / gx));
}

ur_status ur_batch_launch_sigma(const BatchSigmaItem* items, int count, int maxnb, cudaStream_t s) {
  if (count <= 0) return UR_OK;
  k_batch_sigma<<<dim3((unsigned)((maxnb + 255) / 256), (unsigned)count), 256, 0, s>>>(items);
  UR_LAUNCH_CHECK("k_batch_sigma");
  return UR_OK;
}

ur_status ur_batch_launch_grad(const BatchGradItem* items, const long long* start, int count, long long nblocks,
                               size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return UR_OK;
  UR_REQUIRE(nblocks < (1ll << 31), "batched adjoint rows: too many blocks");
  if (smem > 48 * 1024)
    UR_CUDA_CHECK(cudaFuncSetAttribute(k_batch_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_batch_grad<<<(unsigned)nblocks, 256, smem, s>>>(items, start, count);
  UR_LAUNCH_CHECK("k_batch_grad");
  return UR_OK;
}

// ---------------------------------------------------------------------------
// Out-of-core adjoint (the per-slab adjoint of the streamed forward): the inverse
// intermediate of all N planes does not fit when the grid is large, so the output planes
// are produced slab by slab.  For every slab the z pass is recomputed over all spectrum
// columns from the forward intermediate (F~ along z, times sigma(bin), inverse along z)
// and only the slab's planes are kept; the slab then goes through the y inverse and the
// row pass (dL/du accumulated, dL/dm written to a device staging buffer and copied to
// pinned host memory on a copy stream, double-buffered).
// ---------------------------------------------------------------------------
extern "C" ur_status ur_plan_set_adj_slab_planes(ur_plan* p, int32_t planes) {
  UR_REQUIRE(p && planes >= 1, "ur_plan_set_adj_slab_planes: bad argument");
  p->adj_slab_planes = planes > p->n ? p->n : planes;
  return UR_OK;
}

extern "C" ur_status ur_backward_slabs(const ur_plan* p, const double* dl_dmean, const double* fwd_bins,
                                       const float* cell, int32_t ucell, const int32_t* origin, const ur_shape* shape,
                                       const float* weights, float* dl_dcell, float* dl_dmask_host, void* ws,
                                       size_t ws_bytes, void* stream) {
  UR_REQUIRE(p && dl_dmean && fwd_bins && cell && shape && dl_dcell && ws, "ur_backward_slabs: null argument");
  UR_REQUIRE(p->fast, "ur_backward_slabs: power-of-two grids only (edge %d)", p->n);
  UR_REQUIRE(ucell >= 1, "ur_backward_slabs: empty cell");
  UR_REQUIRE(!origin || (origin[0] >= 0 && origin[1] >= 0 && origin[2] >= 0), "ur_backward_slabs: origin must be >= 0");
  UR_REQUIRE(shape->kind >= UR_SHAPE_SPHERE && shape->kind <= UR_SHAPE_WEIGHTS, "ur_backward_slabs: bad shape kind");
  UR_REQUIRE(shape->kind != UR_SHAPE_WEIGHTS || weights, "ur_backward_slabs: weights required for UR_SHAPE_WEIGHTS");
  UR_REQUIRE(!weights || ((uintptr_t)weights % 8) == 0, "ur_backward_slabs: weights must be 8-byte aligned");
  const size_t need = ur_workspace_size(p, UR_WS_FORWARD | UR_WS_ADJ_SLABS);
  UR_REQUIRE(ws_bytes >= need, "ur_backward_slabs: workspace %zu < %zu bytes", ws_bytes, need);
  UR_REQUIRE(((uintptr_t)ws % 256) == 0, "ur_backward_slabs: misaligned ws");
  if (p->vsinc) {
    ur_set_error("ur_backward_slabs: the adjoint of the voxel-sinc corrected binning is not built");
    return UR_ERR_UNSUPPORTED;
  }
  if (dl_dmask_host) {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, dl_dmask_host);
    UR_REQUIRE(e == cudaSuccess && at.type == cudaMemoryTypeHost,
               "ur_backward_slabs: dl_dmask_host must be page-locked host memory");
  }
  UR_TRY(ur_fault_point("backward"));
  cudaStream_t s = (cudaStream_t)stream;
  const int n = p->n, H = p->H, nb = p->nbins, S = p->adj_slab_planes;
  const double n3 = (double)n * n * n;
  // workspace: [X][two host staging slabs][Y slab][sigma][two dL/dm staging slabs of SM planes]
  const int SM = ur_adj_dm_planes(p);
  float2* X = (float2*)ws;
  char* o = (char*)ws + ur_align_up(p->ws_inter, 256) + 2 * ur_align_up(p->ws_slab, 256);
  float2* Ys = (float2*)o;
  o += ur_align_up((size_t)S * n * H * sizeof(float2), 256);
  float* sigma = (float*)o;
  o += ur_align_up(p->ws_sigma, 256);
  float* dm[2];
  const size_t dm_bytes = (size_t)SM * n * n * sizeof(float);
  dm[0] = (float*)o;
  dm[1] = (float*)(o + ur_align_up(dm_bytes, 256));

  k_sigma<<<(nb + 255) / 256, 256, 0, s>>>(dl_dmean, fwd_bins, nb, n3, 0, sigma);
  UR_LAUNCH_CHECK("k_sigma");
  UR_CUDA_CHECK(cudaMemsetAsync(dl_dcell, 0, sizeof(float) * (size_t)ucell * ucell * ucell, s));
  const int k2_zero = (int)(p->thr_host[nb] < 0x7fffffff ? p->thr_host[nb] : 0x7fffffff);

  GradArgs g;
  memset(&g, 0, sizeof g);
  g.tw = p->tw;
  g.stw = p->stw + p->stw_m_off;
  g.cell = cell;
  g.ucell = ucell;
  if (origin) {
    g.ox = origin[0] % ucell;
    g.oy = origin[1] % ucell;
    g.oz = origin[2] % ucell;
  }
  g.sh = ur_shape_args(shape);
  g.weights = shape->kind == UR_SHAPE_WEIGHTS ? weights : nullptr;
  g.inv_n3 = (float)(1.0 / n3);
  g.dl_dcell = dl_dcell;

  cudaStream_t cs = nullptr;
  cudaEvent_t done[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  ur_status st = UR_OK;
  if (dl_dmask_host) {
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
      ok = cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      ur_set_error("ur_backward_slabs: cannot create the copy stream or its events");
      st = UR_ERR_CUDA;
    }
  }
  int sub = 0;  // running index of the dL/dm staging sub-slabs (double-buffered)
  for (int za = 0; za < n && st == UR_OK; za += S) {
    const int cnt = za + S <= n ? S : n - za;
    // z pass over every column, keeping planes [za, za + cnt)
    ColArgs a = ur_col_args(p);
    a.ncols = (long long)n * H;
    a.A = H;
    a.S = (long long)n * H;
    a.Ad = H;
    a.Sd = (long long)n * H;
    a.src = X;
    a.nload = p->nz;
    a.zoff = p->z0;
    a.dst = Ys;
    a.sigma = sigma;
    a.k2_zero = k2_zero;
    a.out_lo = za;
    a.out_cnt = cnt;
    ur_timing_begin("adj_cols_z", s);
    st = ur_fast_cols(n, 3 /* z adjoint */, a, s);
    ur_timing_end(s);
    if (st != UR_OK) break;
    // y inverse of the slab, in place
    ColArgs c = ur_col_args(p);
    c.src = Ys;
    c.dst = Ys;
    c.ncols = (long long)cnt * H;
    c.A = (long long)n * H;
    c.S = H;
    c.Ad = c.A;
    c.Sd = c.S;
    c.nload = n;
    c.zoff = 0;
    c.nbins = 0;
    c.k2_zero = k2_zero;
    ur_timing_begin("adj_cols_y", s);
    st = ur_fast_cols(n, 1 /* y inverse */, c, s);
    ur_timing_end(s);
    if (st != UR_OK) break;
    // rows of the slab in sub-slabs of SM planes: dL/du accumulated, dL/dm into staging buffer b
    for (int zb = za; zb < za + cnt && st == UR_OK; zb += (dl_dmask_host ? SM : cnt), ++sub) {
      const int cz = dl_dmask_host ? (zb + SM <= za + cnt ? SM : za + cnt - zb) : cnt;
      const int b = sub & 1;
      if (dl_dmask_host && sub >= 2) cudaStreamWaitEvent(s, freed[b], 0);
      g.Y = Ys;
      g.ybase_z = za;
      g.z0 = zb;
      g.dl_dmask = dl_dmask_host ? dm[b] : nullptr;
      g.mbase_z = zb;
      ur_timing_begin("adj_rows_grad", s);
      st = ur_fast_rows_grad(n, g, cz, s);
      ur_timing_end(s);
      if (st != UR_OK) break;
      if (dl_dmask_host) {
        cudaEventRecord(done[b], s);
        cudaStreamWaitEvent(cs, done[b], 0);
        const cudaError_t ce = cudaMemcpyAsync(dl_dmask_host + (size_t)zb * n * n, dm[b], (size_t)cz * n * n * sizeof(float),
                                               cudaMemcpyDeviceToHost, cs);
        if (ce != cudaSuccess) {
          ur_set_error("ur_backward_slabs: dL/dm copy failed: %s", cudaGetErrorString(ce));
          st = UR_ERR_CUDA;
          break;
        }
        cudaEventRecord(freed[b], cs);
      }
    }
  }
  if (cs) {
    // the caller's stream waits for the copies still queued
    cudaEvent_t end;
    if (cudaEventCreateWithFlags(&end, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(end, cs);
      cudaStreamWaitEvent(s, end, 0);
      cudaEventDestroy(end);
    }
    cudaStreamDestroy(cs);
  }
  for (int b = 0; b < 2; ++b) {
    if (done[b]) cudaEventDestroy(done[b]);
    if (freed[b]) cudaEventDestroy(freed[b]);
  }
  return st;
}
