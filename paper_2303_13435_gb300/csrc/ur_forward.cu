// Forward path: Sec. 2.4 separated transform (Eq. 2) and Sec. 2.5 Q binning.
//
//   pass 1a  k_rows_r2c        real-to-complex transform along x of every row of
//                              the planes that hold density (two reals packed as
//                              one complex, N/2-point FFT, then the split step)
//   pass 1b  k_cols<COL_Y>     complex transform along y of each (plane, kx)
//                              column, in place: with 1a, the 2D transform of
//                              every nonzero plane (inner sum of Eq. 2)
//   pass 2   k_cols<COL_ZBIN>  complex transform along z of each (ky, kx)
//                              column; planes outside [z0, z0+nz) enter as zeros
//                              (Sec. 2.4: skipped slices are padded); |F|^2 and
//                              the Q-bin sums are taken from shared memory
//   k_finalize                 per-bin counts, sums, mean and standard error
//
// Layouts: intermediate X[p][y][kx] (p = plane - z0), complex64, kx contiguous,
// N/2+1 per row.  Columns of pass 1b are c = p*(N/2+1) + kx; columns of pass 2
// are c = ky_index*(N/2+1) + kx.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "ur_fast.cuh"

#define BIN_CHUNK 8  // consecutive |kz| per thread in the binning walk

// ---------------------------------------------------------------------------
// Pass 1a
// Row r (r = p*N + y) holds N reals read as N/2 complex z[m] = (x[2m], x[2m+1]);
// Z = FFT_{N/2}(z); then, with Z[M] = Z[0],
//   X[k] = (Z[k] + conj Z[M-k])/2 - i W_N^k (Z[k] - conj Z[M-k])/2,  k = 0..M,
// which recombines the transforms of the even and the odd samples.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float2 load_pair(const T* p);
template <>
__device__ __forceinline__ float2 load_pair<float>(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
template <>
__device__ __forceinline__ float2 load_pair<__half>(const __half* p) {
  __half2 h = __ldg(reinterpret_cast<const __half2*>(p));
  return __half22float2(h);
}

struct NoLd {
  __device__ __forceinline__ float2 operator()(int, int) const { return make_float2(0.f, 0.f); }
};
struct NoSt {
  __device__ __forceinline__ void operator()(int, int, float2) const {}
};

// GEN = 1: the row's density is generated here (Sec. 2.3 tile + mask) instead of read.
// Body of one block (block index blk); shared by the single-plan and batched launches.
template <int GEN, typename T>
__device__ __forceinline__ void rows_r2c_body(const RowArgs& ra, int N, int RB, const StageInfo* __restrict__ sched,
                                              int nst, long long blk) {
  extern __shared__ float2 smem[];
  const T* __restrict__ ed = reinterpret_cast<const T*>(ra.ed);
  float2* __restrict__ X = ra.X;
  const long long nrows = ra.nrows;
  const float2* __restrict__ tw = ra.tw;
  const int M = N >> 1, H = M + 1;
  const long long r0 = blk * RB;
  const FastDiv dm((uint32_t)M), dh((uint32_t)H);
  // generated rows: row r = p N + y (r < 2^31) and the cell indices, by multiply-shift
  const FastDiv dn((uint32_t)N), du((uint32_t)(GEN ? ra.ucell : 1));
  for (int f = threadIdx.x; f < RB * M; f += blockDim.x) {
    const int t = (int)dm.div((uint32_t)f);
    const int m = f - t * M;
    const long long r = r0 + t;
    float2 v = make_float2(0.f, 0.f);
    if (r < nrows) {
      if (GEN) {
        const int p = (int)dn.div((uint32_t)r), y = (int)r - p * N, z = ra.z0 + p, x = 2 * m, U = ra.ucell;
        const float* crow =
            ra.cell + ((long long)du.mod((uint32_t)(z + ra.oz)) * U + du.mod((uint32_t)(y + ra.oy))) * U;
        float m0, m1;
        if (ra.weights) {
          const float2 mw = __ldg(reinterpret_cast<const float2*>(ra.weights + ((long long)z * N + y) * N + x));
          m0 = mw.x;
          m1 = mw.y;
        } else {
          m0 = mask_at(ra.sh, x, y, z);
          m1 = mask_at(ra.sh, x + 1, y, z);
        }
        if (GEN == 2)
          v = make_float2(__fmul_rn(lattice_sample(ra.lat, ra.sh, ra.cell, U, x, y, z), m0),
                          __fmul_rn(lattice_sample(ra.lat, ra.sh, ra.cell, U, x + 1, y, z), m1));
        else
          v = make_float2(__fmul_rn(__ldg(crow + du.mod((uint32_t)(x + ra.ox))), m0),
                          __fmul_rn(__ldg(crow + du.mod((uint32_t)(x + 1 + ra.ox))), m1));
      } else {
        v = load_pair<T>(ed + r * N + 2 * m);
      }
    }
    smem[f] = v;
  }
  __syncthreads();
  fft_lines<false, UR_EMAX>(smem, M, RB, sched, nst, tw);
  for (int f = threadIdx.x; f < RB * H; f += blockDim.x) {
    const int t = (int)dh.div((uint32_t)f);
    const int k = f - t * H;
    const long long r = r0 + t;
    if (r >= nrows) continue;
    const float2* Z = smem + t * M;
    const float2 zk = Z[k == M ? 0 : k];
    const float2 zc = cconj(Z[k == 0 ? 0 : M - k]);
    const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
    const float2 d = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
    const float2 o = make_float2(d.y, -d.x);  // -i d
    const float2 w = __ldg(tw + k);
    X[r * H + k] = cadd(e, cmul(w, o));
  }
}

template <int GEN, typename T>
__global__ void __launch_bounds__(256, 4) k_rows_r2c(RowArgs ra, int N, int RB, const StageInfo* __restrict__ sched,
                                                     int nst) {
  rows_r2c_body<GEN, T>(ra, N, RB, sched, nst, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Column passes.  A block owns TX consecutive columns; column c of the source
// has elements src[(c / H) * A + c % H + i * S], i < nload, placed at shared
// position zoff + i (all other positions zero).
// ---------------------------------------------------------------------------
// Column indices stay below 2^31 (at most N (N/2+1) columns), so the block's
// index arithmetic runs in 32 bits with multiply-shift division (FastDiv).
struct ColDivs {
  FastDiv tx, h;
  __device__ explicit ColDivs(const ColArgs& a) : tx((uint32_t)a.TX), h((uint32_t)a.H) {}
};

__device__ __forceinline__ long long col_offset(uint32_t c, const FastDiv& dh, long long A) {
  const uint32_t o = dh.div(c);
  return (long long)o * A + (c - o * dh.d);
}

__device__ __forceinline__ void load_columns(const ColArgs& a, const ColDivs& dv, float2* buf, long long c0, int N) {
  const int TX = a.TX;
  for (int f = threadIdx.x; f < TX * N; f += blockDim.x) {
    const int i = (int)dv.tx.div((uint32_t)f);
    const int t = f - i * TX;
    const long long c = c0 + t;
    const int li = i - a.zoff;
    float2 v = make_float2(0.f, 0.f);
    if (c < a.ncols && li >= 0 && li < a.nload) {
      v = __ldg(a.src + col_offset((uint32_t)c, dv.h, a.A) + (long long)li * a.S);
    }
    buf[t * a.pitch + i] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ void store_columns(const ColArgs& a, const ColDivs& dv, const float2* buf, long long c0,
                                              int N) {
  const int TX = a.TX;
  for (int f = threadIdx.x; f < TX * N; f += blockDim.x) {
    const int i = (int)dv.tx.div((uint32_t)f);
    const int t = f - i * TX;
    const long long c = c0 + t;
    if (c < a.ncols) a.dst[col_offset((uint32_t)c, dv.h, a.Ad) + (long long)i * a.Sd] = buf[t * a.pitch + i];
  }
}

// Element access of the first and last transform stages (fft_lines_io): element i of
// tile line `line` (column c0 + line) in the source or destination layout.
struct ColLd {
  const float2* src;
  long long A, S, ncols, c0;
  int zoff, nload;
  FastDiv h;
  __device__ ColLd(const ColArgs& a, const ColDivs& dv, long long c)
      : src(a.src), A(a.A), S(a.S), ncols(a.ncols), c0(c), zoff(a.zoff), nload(a.nload), h(dv.h) {}
  __device__ __forceinline__ float2 operator()(int line, int i) const {
    const long long c = c0 + line;
    const int li = i - zoff;
    if (c < ncols && li >= 0 && li < nload) return __ldg(src + col_offset((uint32_t)c, h, A) + (long long)li * S);
    return make_float2(0.f, 0.f);
  }
};
struct ColSt {
  float2* dst;
  long long Ad, Sd, ncols, c0;
  FastDiv h;
  __device__ ColSt(const ColArgs& a, const ColDivs& dv, long long c)
      : dst(a.dst), Ad(a.Ad), Sd(a.Sd), ncols(a.ncols), c0(c), h(dv.h) {}
  __device__ __forceinline__ void operator()(int line, int i, float2 v) const {
    const long long c = c0 + line;
    if (c < ncols) dst[col_offset((uint32_t)c, h, Ad) + (long long)i * Sd] = v;
  }
};

// Walk the (column, |kz|) pairs of the block's spectrum columns in chunks of
// BIN_CHUNK consecutive |kz| = m.  k^2 = kx^2 + ky^2 + m^2 grows with m, so the
// bin index only moves forward inside a chunk.  kz = m and kz = N - m share k^2.
// Op(t, m, bin, weight) is called for every pair.
template <typename Op>
__device__ __forceinline__ void walk_bins(const ColArgs& a, const ColDivs& dv, const int32_t* __restrict__ thr,
                                          long long c0, Op op) {
  const int M = a.M, H = a.H, N = a.N;
  const int nch = (H + BIN_CHUNK - 1) / BIN_CHUNK;
  const int ntask = a.TX * nch;
  const FastDiv dch((uint32_t)nch);
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    const int t = (int)dch.div((uint32_t)task);
    const int ch = task - t * nch;
    const long long c = c0 + t;
    if (c >= a.ncols) continue;
    const int kyi = (int)dv.h.div((uint32_t)c);
    const int kx = (int)c - kyi * H;
    const int ky = kyi < M ? kyi : kyi - N;
    const int c2 = kx * kx + ky * ky;
    const float w = (kx == 0 || kx == M) ? 1.f : 2.f;
    const int m0 = ch * BIN_CHUNK;
    const int m1 = min(m0 + BIN_CHUNK, M + 1);
    int cur = bin_search(thr, a.nbins, c2 + m0 * m0);
    // voxel-sinc factor of the column (kx, ky); the kz part is applied per element
    const float cs = a.vs ? __ldg(a.vs + kx) * __ldg(a.vs + (ky < 0 ? -ky : ky)) : 1.f;
    op.begin(cur, cs);
    for (int m = m0; m < m1; ++m) {
      const int s = c2 + m * m;
      while (cur < a.nbins && thr[cur + 1] <= s) ++cur;
      op.visit(t, m, cur, w);
    }
    op.end(w);
  }
}

struct BinAccum {
  const float2* buf;
  int pitch, M, N, nbins;
  float iscale;
  double* hs;
  double* hs2;
  int run;
  float aI, aI2;
  const float* vs;
  float cs;
  __device__ __forceinline__ void flush(float w) {
    if (run >= 0 && run < nbins && (aI != 0.f || aI2 != 0.f)) {
      atomicAdd(hs + run, (double)(w * aI));
      atomicAdd(hs2 + run, (double)(w * aI2));
    }
    aI = 0.f;
    aI2 = 0.f;
  }
  __device__ __forceinline__ void begin(int b, float c) {
    run = b;
    aI = 0.f;
    aI2 = 0.f;
    cs = c;
  }
  __device__ __forceinline__ void visit(int t, int m, int b, float w) {
    if (b != run) {
      flush(w);
      run = b;
    }
    const float sc = vs ? iscale * (cs * __ldg(vs + m)) : iscale;
    const float2 f1 = buf[t * pitch + m];
    const float i1 = (f1.x * f1.x + f1.y * f1.y) * sc;
    float s = i1, s2 = i1 * i1;
    if (m != 0 && m != M) {
      const float2 f2 = buf[t * pitch + N - m];
      const float i2 = (f2.x * f2.x + f2.y * f2.y) * sc;
      s += i2;
      s2 += i2 * i2;
    }
    aI += s;
    aI2 += s2;
  }
  __device__ __forceinline__ void end(float w) { flush(w); }
};

struct SigmaScale {
  float2* buf;
  int pitch, M, N, nbins;
  const float* sigma;
  __device__ __forceinline__ void begin(int, float) {}
  __device__ __forceinline__ void end(float) {}
  __device__ __forceinline__ void visit(int t, int m, int b, float) {
    const float sg = (b >= 0 && b < nbins) ? __ldg(sigma + b) : 0.f;
    float2* col = buf + t * pitch;
    col[m] = cscale(col[m], sg);
    if (m != 0 && m != M) col[N - m] = cscale(col[N - m], sg);
  }
};

// One block per tile of TX columns.  (A persistent loop over tiles around the
// shared-memory FFT made the compiler spill ~1.3 KB per thread.)
template <int MODE, bool INV>
__device__ __forceinline__ void cols_body(const ColArgs& a, long long blk) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_blo, s_bhi;
  float2* buf = reinterpret_cast<float2*>(smraw);
  const int N = a.N;
  const size_t buf_bytes = ur_align_up_dev((size_t)a.TX * a.pitch * sizeof(float2), 16);
  int32_t* thr = reinterpret_cast<int32_t*>(smraw + buf_bytes);
  double* hs = nullptr;
  double* hs2 = nullptr;
  const long long c0 = blk * a.TX;
  const ColDivs dv(a);
  if (MODE != COL_Y && a.nbins > 0) {
    for (int j = threadIdx.x; j <= a.nbins; j += blockDim.x) thr[j] = __ldg(a.thr + j);
    if (MODE == COL_ZBIN) {
      hs = reinterpret_cast<double*>(smraw + buf_bytes + ur_align_up_dev((size_t)(a.nbins + 1) * 4, 16));
      hs2 = hs + a.nbins;
      if (threadIdx.x == 0) {
        s_blo = 0x7fffffff;
        s_bhi = -1;
      }
    }
  }
  __syncthreads();
  if (MODE == COL_ZBIN && a.nbins > 0) {
    // bins this tile can reach: k^2 in [min kx^2+ky^2, max kx^2+ky^2 + (N/2)^2]
    if (threadIdx.x < a.TX && c0 + threadIdx.x < a.ncols) {
      const long long c = c0 + threadIdx.x;
      const int kyi = (int)dv.h.div((uint32_t)c);
      const int kx = (int)c - kyi * a.H;
      const int ky = kyi < a.M ? kyi : kyi - N;
      const int c2 = kx * kx + ky * ky;
      atomicMin(&s_blo, max(bin_search(thr, a.nbins, c2), 0));
      atomicMax(&s_bhi, min(bin_search(thr, a.nbins, c2 + a.M * a.M), a.nbins - 1));
    }
    __syncthreads();
    for (int j = s_blo + (int)threadIdx.x; j <= s_bhi; j += blockDim.x) {
      hs[j] = 0.0;
      hs2[j] = 0.0;
    }
  }
  {
    // with two or more stages the first stage reads the columns from global memory and, where
    // the result goes back to global memory, the last stage writes it (no staging round trips)
    const bool io = a.nst >= 2;
    if (MODE == COL_Y) {
      if (io) {
        fft_lines_io<INV, UR_EMAX, true, true, true>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw, ColLd(a, dv, c0),
                                               ColSt(a, dv, c0));
      } else {
        load_columns(a, dv, buf, c0, N);
        fft_lines<INV, UR_EMAX>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw);
        store_columns(a, dv, buf, c0, N);
      }
    } else if (MODE == COL_ZBIN) {
      if (io) {
        fft_lines_io<false, UR_EMAX, true, false, true>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw, ColLd(a, dv, c0), NoSt());
      } else {
        load_columns(a, dv, buf, c0, N);
        fft_lines<false, UR_EMAX>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw);
      }
      if (a.fout) {
        for (int f = threadIdx.x; f < a.TX * N; f += blockDim.x) {
          const int i = (int)dv.tx.div((uint32_t)f);
          const int t = f - i * a.TX;
          const long long c = c0 + t;
          if (c < a.ncols) a.fout[(long long)i * N * a.H + c] = cscale(buf[t * a.pitch + i], a.fscale);
        }
      }
      if (a.nbins > 0) {
        BinAccum acc{buf, a.pitch, a.M, N, a.nbins, a.iscale, hs, hs2, -1, 0.f, 0.f, a.vs, 1.f};
        walk_bins(a, dv, thr, c0, acc);
      }
    } else {  // COL_ZADJ: F along z (recomputed or given), times sigma(bin), inverse along z
      if (io && !a.skip_fwd) {
        fft_lines_io<false, UR_EMAX, true, false, true>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw, ColLd(a, dv, c0), NoSt());
      } else {
        load_columns(a, dv, buf, c0, N);
        if (!a.skip_fwd) fft_lines<false, UR_EMAX>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw);
      }
      SigmaScale sc{buf, a.pitch, a.M, N, a.nbins, a.sigma};
      walk_bins(a, dv, thr, c0, sc);
      __syncthreads();
      if (io) {
        fft_lines_io<true, UR_EMAX, false, true, true>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw, NoLd(), ColSt(a, dv, c0));
      } else {
        fft_lines<true, UR_EMAX>(buf, a.pitch, a.TX, a.sched, a.nst, a.tw);
        store_columns(a, dv, buf, c0, N);
      }
    }
  }
  if (MODE == COL_ZBIN && a.nbins > 0) {
    __syncthreads();
    for (int j = s_blo + (int)threadIdx.x; j <= s_bhi; j += blockDim.x) {
      if (hs[j] != 0.0) atomicAdd(a.gsum + j, hs[j]);
      if (hs2[j] != 0.0) atomicAdd(a.gsum2 + j, hs2[j]);
    }
  }
}

template <int MODE, bool INV>
__global__ void __launch_bounds__(256, 4) k_cols(ColArgs a) {
  cols_body<MODE, INV>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Finalize: bins[UR_BIN_FIELDS][B] from the accumulated sums (in I' units:
// I' = N^3 I) and the plan's per-bin count and sum |Q|.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_bin(double* __restrict__ bins, const double* __restrict__ geo, int nb,
                                             double inv_n3, int j) {
  if (j >= nb) return;
  const double n = geo[j];
  const double s = bins[UR_BIN_SUM_I * nb + j] * inv_n3;
  const double s2 = bins[UR_BIN_SUM_I2 * nb + j] * (inv_n3 * inv_n3);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  bins[UR_BIN_COUNT * nb + j] = n;
  bins[UR_BIN_SUM_I * nb + j] = s;
  bins[UR_BIN_SUM_I2 * nb + j] = s2;
  bins[UR_BIN_SUM_Q * nb + j] = geo[nb + j];
  double mean = nan, sem = nan;
  if (n > 0) mean = s / n;
  if (n > 1) {
    double var = (s2 - s * mean) / (n - 1.0);
    if (var < 0) var = 0;
    sem = sqrt(var / n);
  }
  bins[UR_BIN_MEAN * nb + j] = mean;
  bins[UR_BIN_SEM * nb + j] = sem;
}

__global__ void k_finalize(double* __restrict__ bins, const double* __restrict__ geo, int nb, double inv_n3) {
  finalize_bin(bins, geo, nb, inv_n3, blockIdx.x * blockDim.x + threadIdx.x);
}

// finalize of the power-of-two column pass, which leaves shifted sums (ur_bin_shift)
__global__ void k_finalize_shifted(double* __restrict__ bins, const double* __restrict__ geo, int nb, double inv_n3) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nb) ur_finalize_shifted(bins, geo, nb, inv_n3, j);
}

// ---------------------------------------------------------------------------
// Plan-time bin geometry: count (weighted by the half-spectrum multiplicity)
// and sum of |Q| per bin over the full N^3 grid; independent of the data.
// One thread per (ky, kx) column, walking |kz| = m; block histogram in shared
// memory, then one global add per touched bin.
// ---------------------------------------------------------------------------
__global__ void k_geometry(const int32_t* __restrict__ thr_g, int nb, int N, double dq,
                           unsigned long long* __restrict__ gcount, double* __restrict__ gsumq) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int32_t* thr = reinterpret_cast<int32_t*>(smraw);
  unsigned long long* hc = reinterpret_cast<unsigned long long*>(smraw + ur_align_up_dev((size_t)(nb + 1) * 4, 16));
  double* hq = reinterpret_cast<double*>(hc + nb);
  for (int j = threadIdx.x; j <= nb; j += blockDim.x) thr[j] = thr_g[j];
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    hc[j] = 0ull;
    hq[j] = 0.0;
  }
  __syncthreads();
  const int M = N / 2, H = M + 1;
  const long long ncols = (long long)N * H;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += (long long)gridDim.x * blockDim.x) {
    const int kyi = (int)(c / H);
    const int kx = (int)(c - (long long)kyi * H);
    const int ky = kyi < M ? kyi : kyi - N;
    const int c2 = kx * kx + ky * ky;
    const unsigned long long w = (kx == 0 || kx == M) ? 1ull : 2ull;
    int cur = bin_search(thr, nb, c2);
    int run = cur;
    unsigned long long cnt = 0;
    double sq = 0.0;
    for (int m = 0; m <= M; ++m) {
      const int s = c2 + m * m;
      while (cur < nb && thr[cur + 1] <= s) ++cur;
      if (cur != run) {
        if (run >= 0 && run < nb && cnt) {
          atomicAdd(hc + run, cnt * w);
          atomicAdd(hq + run, sq * (double)w);
        }
        run = cur;
        cnt = 0;
        sq = 0.0;
      }
      const unsigned long long mult = (m == 0 || m == M) ? 1ull : 2ull;
      cnt += mult;
      sq += (double)mult * sqrt((double)s);
    }
    if (run >= 0 && run < nb && cnt) {
      atomicAdd(hc + run, cnt * w);
      atomicAdd(hq + run, sq * (double)w);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    if (hc[j]) {
      atomicAdd(gcount + j, hc[j]);
      atomicAdd(gsumq + j, hq[j] * dq);
    }
  }
}

__global__ void k_geo_to_double(const unsigned long long* __restrict__ c, double* __restrict__ out, int nb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nb) out[j] = (double)c[j];
}

__global__ void k_binlut(const int32_t* __restrict__ thr, int nb, int smax, int16_t* __restrict__ lut) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > smax) return;
  const int b = bin_search(thr, nb, s);
  lut[s] = (int16_t)((b >= 0 && b < nb) ? b : -1);
}

__global__ void k_bincoarse(const int32_t* __restrict__ thr, int nb, int shift, int16_t* __restrict__ crs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < UR_COARSE_ENTRIES) crs[i] = (int16_t)bin_search(thr, nb, i << shift);
}

ur_status ur_launch_geometry(ur_plan* p, cudaStream_t s) {
  {
    const int smax = 3 * (p->n / 2) * (p->n / 2);
    int sh = 0;
    while ((smax >> sh) >= UR_COARSE_ENTRIES) ++sh;
    p->coarse_shift = sh;
    UR_CUDA_CHECK(cudaMalloc(&p->binlut, sizeof(int16_t) * ((size_t)smax + 1)));
    k_binlut<<<(smax + 256) / 256, 256, 0, s>>>(p->thr, p->nbins, smax, p->binlut);
    UR_LAUNCH_CHECK("k_binlut");
    UR_CUDA_CHECK(cudaMalloc(&p->bincoarse, sizeof(int16_t) * UR_COARSE_ENTRIES));
    k_bincoarse<<<(UR_COARSE_ENTRIES + 255) / 256, 256, 0, s>>>(p->thr, p->nbins, sh, p->bincoarse);
    UR_LAUNCH_CHECK("k_bincoarse");
  }
  const int nb = p->nbins;
  unsigned long long* cnt = nullptr;
  UR_CUDA_CHECK(cudaMalloc(&cnt, sizeof(unsigned long long) * nb));
  UR_CUDA_CHECK(cudaMemset(cnt, 0, sizeof(unsigned long long) * nb));
  UR_CUDA_CHECK(cudaMemset(p->geo, 0, sizeof(double) * 2 * nb));
  const size_t smem = ur_align_up((size_t)(nb + 1) * 4, 16) + (size_t)nb * 16;
  if (smem > 48 * 1024) UR_CUDA_CHECK(cudaFuncSetAttribute(k_geometry, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long ncols = (long long)p->n * p->H;
  long long blocks = (ncols + 255) / 256;
  const long long cap = (long long)p->num_sms * 4;
  if (blocks > cap) blocks = cap;
  k_geometry<<<(int)blocks, 256, smem, s>>>(p->thr, nb, p->n, p->dq, cnt, p->geo + nb);
  UR_LAUNCH_CHECK("k_geometry");
  k_geo_to_double<<<(nb + 255) / 256, 256, 0, s>>>(cnt, p->geo, nb);
  UR_LAUNCH_CHECK("k_geo_to_double");
  UR_CUDA_CHECK(cudaStreamSynchronize(s));
  UR_CUDA_CHECK(cudaFree(cnt));
  return UR_OK;
}

// ---------------------------------------------------------------------------
// Standalone binning of a stored half-spectrum intensity (Sec. 2.5)
// ---------------------------------------------------------------------------
__global__ void k_bin_half(const float* __restrict__ I, int N, const int32_t* __restrict__ thr_g, int nb,
                           double* __restrict__ gsum, double* __restrict__ gsum2, double scale,
                           const float* __restrict__ vs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int32_t* thr = reinterpret_cast<int32_t*>(smraw);
  double* hs = reinterpret_cast<double*>(smraw + ur_align_up_dev((size_t)(nb + 1) * 4, 16));
  double* hs2 = hs + nb;
  for (int j = threadIdx.x; j <= nb; j += blockDim.x) thr[j] = thr_g[j];
  for (int j = threadIdx.x; j < 2 * nb; j += blockDim.x) hs[j] = 0.0;
  __syncthreads();
  const int M = N / 2, H = M + 1;
  const long long total = (long long)N * N * H;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e % ((long long)N * H);
    const int kzi = (int)(e / ((long long)N * H));
    const int kyi = (int)(c / H);
    const int kx = (int)(c - (long long)kyi * H);
    const int ky = kyi < M ? kyi : kyi - N;
    const int kz = kzi < M ? kzi : kzi - N;
    const int s = kx * kx + ky * ky + kz * kz;
    const int b = bin_search(thr, nb, s);
    if (b >= 0 && b < nb) {
      const double w = (kx == 0 || kx == M) ? 1.0 : 2.0;
      double v = (double)I[e] * scale;
      if (vs) v *= (double)(__ldg(vs + kx) * __ldg(vs + (ky < 0 ? -ky : ky)) * __ldg(vs + (kz < 0 ? -kz : kz)));
      atomicAdd(hs + b, w * v);
      atomicAdd(hs2 + b, w * v * v);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    if (hs[j] != 0.0) atomicAdd(gsum + j, hs[j]);
    if (hs2[j] != 0.0) atomicAdd(gsum2 + j, hs2[j]);
  }
}

// ---------------------------------------------------------------------------
// Host: kernel configuration for a plan
// ---------------------------------------------------------------------------
size_t ur_colbin_smem(const ur_plan* p) {
  return ur_align_up((size_t)p->col_tx * (p->n + 1) * sizeof(float2), 16) + ur_align_up((size_t)(p->nbins + 1) * 4, 16) +
         (size_t)p->nbins * 16;
}

ur_status ur_configure_kernels(ur_plan* p) {
  const int n = p->n, M = p->M;
  // rows: RB rows of M complex per block, 256 threads, <= EMAX elements per thread
  p->row_threads = 256;
  p->row_rb = (UR_EMAX * p->row_threads) / M;
  if (p->row_rb > 64) p->row_rb = 64;
  if (p->row_rb < 1) p->row_rb = 1;
  p->row_smem = (size_t)p->row_rb * M * sizeof(float2);
  // columns: TX columns of N complex per block
  p->col_threads = 256;
  p->col_tx = (UR_EMAX * p->col_threads) / n;
  if (p->col_tx > 64) p->col_tx = 64;
  if (p->col_tx < 1) p->col_tx = 1;
  p->col_smem = ur_align_up((size_t)p->col_tx * (n + 1) * sizeof(float2), 16) + ur_align_up((size_t)(p->nbins + 1) * 4, 16);
  p->colbin_smem = ur_colbin_smem(p);
  if (p->colbin_smem > 227 * 1024) {
    ur_set_error("ur_plan_create: %d bins need %zu bytes of shared memory per block (max 227 KB)", p->nbins, p->colbin_smem);
    return UR_ERR_UNSUPPORTED;
  }
  // the runtime-radix kernels accept any tile shape up to the per-block limit
  // (ur_plan_set_tiles may change it), so they get the largest dynamic size once
  const int kMaxDyn = 200 * 1024;
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_rows_r2c<0, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_rows_r2c<0, __half>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_rows_r2c<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_rows_r2c<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_cols<COL_Y, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_cols<COL_Y, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_cols<COL_ZBIN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  UR_CUDA_CHECK(cudaFuncSetAttribute(k_cols<COL_ZADJ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
  const long long ntiles = ((long long)n * p->H + p->col_tx - 1) / p->col_tx;
  p->zbin_grid = (int)ntiles;
  // device copy of the radix schedules
  UR_CUDA_CHECK(cudaMalloc(&p->d_sched, sizeof(StageInfo) * 2 * UR_MAX_STAGES));
  UR_CUDA_CHECK(cudaMemcpy(p->d_sched, p->sched_n.st, sizeof(StageInfo) * UR_MAX_STAGES, cudaMemcpyHostToDevice));
  UR_CUDA_CHECK(cudaMemcpy(p->d_sched + UR_MAX_STAGES, p->sched_m.st, sizeof(StageInfo) * UR_MAX_STAGES, cudaMemcpyHostToDevice));
  // workspace regions
  p->ws_inter = (size_t)p->nz * n * p->H * sizeof(float2);
  p->ws_inv = (size_t)n * n * p->H * sizeof(float2);
  p->ws_sigma = (size_t)p->nbins * sizeof(float);
  // host-resident ED: slabs of about 256 MiB, two of them in the workspace
  {
    const size_t ed_plane = (size_t)n * n * (p->ed_dtype == UR_F16 ? 2 : 4);
    long long sp = (long long)((256ull << 20) / ed_plane);
    if (sp < 1) sp = 1;
    if (sp > p->nz) sp = p->nz;
    p->slab_planes = (int)sp;
    p->ws_slab = (size_t)sp * ed_plane;
  }
  // out-of-core adjoint: about 4 GiB of inverse intermediate per slab
  {
    long long ap = (long long)((4ull << 30) / ((size_t)n * p->H * sizeof(float2)));
    if (ap < 1) ap = 1;
    if (ap > n) ap = n;
    p->adj_slab_planes = (int)ap;
  }
  // power-of-two kernels; by default every pass runs over all planes at once
  // (ur_plan_set_chunk_planes can split the plane pass and the adjoint's y and
  // row passes into chunks whose intermediate stays in L2 between the two
  // kernels; on the 512^3 workload one launch per pass measured faster)
  p->fast = ur_fast_supported(n) ? 1 : 0;
  p->chunk_planes = n;
  p->ws_chunk = 0;
  return UR_OK;
}

ur_status ur_launch_cols(int mode, bool inv, const ur_plan* p, const ColArgs& a, int grid, size_t smem, cudaStream_t s) {
  (void)p;
  if (grid <= 0) return UR_OK;
  if (mode == COL_Y && !inv) k_cols<COL_Y, false><<<grid, p->col_threads, smem, s>>>(a);
  else if (mode == COL_Y) k_cols<COL_Y, true><<<grid, p->col_threads, smem, s>>>(a);
  else if (mode == COL_ZBIN) k_cols<COL_ZBIN, false><<<grid, p->col_threads, smem, s>>>(a);
  else k_cols<COL_ZADJ, false><<<grid, p->col_threads, smem, s>>>(a);
  UR_LAUNCH_CHECK("k_cols");
  return UR_OK;
}

ColArgs ur_col_args(const ur_plan* p) {
  ColArgs a;
  memset(&a, 0, sizeof a);
  a.N = p->n;
  a.H = p->H;
  a.M = p->M;
  a.TX = p->col_tx;
  a.pitch = p->n + 1;
  a.sched = p->d_sched;
  a.nst = p->sched_n.nst;
  a.tw = p->tw;
  a.stw = p->stw;
  a.thr = p->thr;
  a.lut = p->binlut;
  a.k2_zero = 0x7fffffff;
  a.vs = p->vsinc;
  a.crs = p->bincoarse;
  a.crs_shift = p->coarse_shift;
  a.nbins = p->nbins;
  return a;
}

// Pass 1 (rows along x, then columns along y) of nplanes planes into X (same
// plane order).  ra carries either the density rows (GEN = 0) or the density
// description (GEN = 1, rows generated in the kernel); ra.z0 is the absolute
// plane of X's first plane.  On the power-of-two path the planes go in chunks
// whose intermediate stays in L2 between the two kernels.
static ur_status plane_pass(const ur_plan* p, RowArgs ra, int gen, long long nplanes, float2* X, cudaStream_t s) {
  const int n = p->n, H = p->H;
  const long long step = p->fast ? p->chunk_planes : nplanes;
  for (long long p0 = 0; p0 < nplanes; p0 += step) {
    const long long np = (p0 + step <= nplanes) ? step : nplanes - p0;
    RowArgs r = ra;
    r.stw = p->stw ? p->stw + p->stw_m_off : nullptr;
    r.fu = FastDiv((uint32_t)(ra.ucell > 0 ? ra.ucell : 1));
    r.X = X + p0 * n * H;
    r.nrows = np * n;
    r.z0 = ra.z0 + (int)p0;
    if (!gen) r.ed = (const char*)ra.ed + p0 * (long long)n * n * (p->ed_dtype == UR_F16 ? 2 : 4);
    // generated sphere on rows of at most one warp: the row pass leaves the rows outside the
    // particle unwritten and the y pass reads them as zeros
    const bool skip = gen && p->fast && n <= 512 && ra.sh.kind == UR_SHAPE_SPHERE && !ra.weights;
    r.skip_empty = skip ? 1 : 0;
    ur_timing_begin("rows_r2c", s);
    if (p->fast) {
      UR_TRY(ur_fast_rows(n, r, gen, p->ed_dtype == UR_F16, s));
    } else {
      const int grid_rows = (int)((r.nrows + p->row_rb - 1) / p->row_rb);
      const StageInfo* sm = p->d_sched + UR_MAX_STAGES;
      if (gen == 2) k_rows_r2c<2, float><<<grid_rows, p->row_threads, p->row_smem, s>>>(r, n, p->row_rb, sm, p->sched_m.nst);
      else if (gen) k_rows_r2c<1, float><<<grid_rows, p->row_threads, p->row_smem, s>>>(r, n, p->row_rb, sm, p->sched_m.nst);
      else if (p->ed_dtype == UR_F32)
        k_rows_r2c<0, float><<<grid_rows, p->row_threads, p->row_smem, s>>>(r, n, p->row_rb, sm, p->sched_m.nst);
      else k_rows_r2c<0, __half><<<grid_rows, p->row_threads, p->row_smem, s>>>(r, n, p->row_rb, sm, p->sched_m.nst);
      UR_LAUNCH_CHECK("k_rows_r2c");
    }
    ur_timing_end(s);
    ColArgs a = ur_col_args(p);
    a.src = r.X;
    a.dst = r.X;
    a.ncols = np * H;
    a.A = (long long)n * H;
    a.S = H;
    a.Ad = a.A;
    a.Sd = a.S;
    a.nload = n;
    a.zoff = 0;
    a.nbins = 0;
    if (skip) {
      a.row_skip = 1;
      a.gen_z0 = r.z0;
      a.sh = ra.sh;
    }
    ur_timing_begin("cols_y", s);
    if (p->fast) {
      UR_TRY(ur_fast_cols(n, 0 /* y forward */, a, s));
    } else {
      const long long ntiles = (a.ncols + a.TX - 1) / a.TX;
      k_cols<COL_Y, false><<<(int)ntiles, p->col_threads, p->col_smem, s>>>(a);
      UR_LAUNCH_CHECK("k_cols<COL_Y>");
    }
    ur_timing_end(s);
  }
  return UR_OK;
}

ur_status ur_plane_pass(const ur_plan* p, const void* ed, long long nplanes, float2* X, cudaStream_t s) {
  RowArgs ra;
  memset(&ra, 0, sizeof ra);
  ra.ed = ed;
  ra.tw = p->tw;
  ra.z0 = p->z0;
  return plane_pass(p, ra, 0, nplanes, X, s);
}

// Pass 2 (+ binning) from the intermediate X holding planes [z0, z0+nz).
ur_status ur_column_pass(const ur_plan* p, const float2* X, double* bins, float2* F_out, cudaStream_t s) {
  const int nb = p->nbins;
  ColArgs a = ur_col_args(p);
  a.src = X;
  a.ncols = (long long)p->n * p->H;
  a.A = p->H;
  a.S = (long long)p->n * p->H;
  a.nload = p->nz;
  a.zoff = p->z0;
  const double n3 = (double)p->n * p->n * p->n;
  a.iscale = (float)(1.0 / n3);
  a.fout = F_out;
  a.fscale = (float)(1.0 / n3);
  if (bins) {
    UR_CUDA_CHECK(cudaMemsetAsync(bins, 0, sizeof(double) * UR_BIN_FIELDS * nb, s));
    a.gsum = bins + UR_BIN_SUM_I * nb;
    a.gsum2 = bins + UR_BIN_SUM_I2 * nb;
    a.gK = ur_shift_slots(bins, nb);
  } else {
    a.nbins = 0;
  }
  // grids of 256 and 512 with binning, when the plan asks for it: the TMA z-column kernel
  const bool zc = bins && p->fast && p->zc_enabled && ur_zcol_supported(p);
  ur_timing_begin("cols_z_bin", s);
  if (zc) {
    UR_TRY(ur_zcol_forward(p, X, bins, F_out, a.iscale, a.fscale, s));
  } else if (p->fast) {
    UR_TRY(ur_fast_cols(p->n, 2 /* z + bins */, a, s));
  } else {
    k_cols<COL_ZBIN, false><<<p->zbin_grid, p->col_threads, p->colbin_smem, s>>>(a);
    UR_LAUNCH_CHECK("k_cols<COL_ZBIN>");
  }
  ur_timing_end(s);
  if (bins && !zc) {  // (the TMA z-column kernel finalizes the bins itself)
    ur_timing_begin("finalize", s);
    if (p->fast) k_finalize_shifted<<<(nb + 255) / 256, 256, 0, s>>>(bins, p->geo, nb, 1.0 / n3);
    else k_finalize<<<(nb + 255) / 256, 256, 0, s>>>(bins, p->geo, nb, 1.0 / n3);
    UR_LAUNCH_CHECK("k_finalize");
    ur_timing_end(s);
  }
  return UR_OK;
}

extern "C" ur_status ur_fft_intensity(const ur_plan* p, const void* ed, int32_t ed_on_host, double* bins, void* F_out,
                                      void* ws, size_t ws_bytes, void* stream) {
  UR_REQUIRE(p && ed && ws, "ur_fft_intensity: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (ed_on_host) return ur_fft_intensity_host(p, ed, bins, (float2*)F_out, ws, ws_bytes, s);
  UR_REQUIRE(ws_bytes >= ur_workspace_size(p, UR_WS_FORWARD), "ur_fft_intensity: workspace %zu < %zu bytes", ws_bytes,
             ur_workspace_size(p, UR_WS_FORWARD));
  UR_REQUIRE(((uintptr_t)ed % 8) == 0 && ((uintptr_t)ws % 256) == 0, "ur_fft_intensity: misaligned ed or ws");
  UR_TRY(ur_fault_point("fft_intensity"));
  float2* X = (float2*)ws;
  UR_TRY(ur_plane_pass(p, ed, p->nz, X, s));
  UR_TRY(ur_column_pass(p, X, bins, (float2*)F_out, s));
  return UR_OK;
}

static ur_status fft_intensity_tiled(const ur_plan* p, const float* cell, int32_t ucell, const int32_t* origin,
                                     const ur_lattice* lattice, const ur_shape* shape, const float* weights,
                                     double* bins, void* F_out, void* ws, size_t ws_bytes, void* stream) {
  UR_REQUIRE(p && cell && shape && ws, "ur_fft_intensity_tiled: null argument");
  UR_REQUIRE(ucell >= 1, "ur_fft_intensity_tiled: empty cell");
  UR_REQUIRE(shape->kind >= UR_SHAPE_SPHERE && shape->kind <= UR_SHAPE_WEIGHTS, "ur_fft_intensity_tiled: bad shape kind");
  UR_REQUIRE(shape->kind != UR_SHAPE_WEIGHTS || weights, "ur_fft_intensity_tiled: weights required for UR_SHAPE_WEIGHTS");
  UR_REQUIRE(!weights || ((uintptr_t)weights % 8) == 0, "ur_fft_intensity_tiled: weights must be 8-byte aligned");
  UR_REQUIRE(ws_bytes >= ur_workspace_size(p, UR_WS_FORWARD), "ur_fft_intensity_tiled: workspace %zu < %zu bytes",
             ws_bytes, ur_workspace_size(p, UR_WS_FORWARD));
  UR_REQUIRE(((uintptr_t)ws % 256) == 0, "ur_fft_intensity_tiled: misaligned ws");
  UR_TRY(ur_fault_point("fft_intensity"));
  cudaStream_t s = (cudaStream_t)stream;
  RowArgs ra;
  memset(&ra, 0, sizeof ra);
  ra.tw = p->tw;
  ra.z0 = p->z0;
  ra.cell = cell;
  ra.ucell = ucell;
  if (origin) {
    UR_REQUIRE(origin[0] >= 0 && origin[1] >= 0 && origin[2] >= 0, "ur_fft_intensity_tiled: origin must be >= 0");
    ra.ox = origin[0];
    ra.oy = origin[1];
    ra.oz = origin[2];
  }
  ra.sh = ur_shape_args(shape);
  ra.lat = ur_lattice_args(lattice);
  ra.weights = shape->kind == UR_SHAPE_WEIGHTS ? weights : nullptr;
  float2* X = (float2*)ws;
  UR_TRY(plane_pass(p, ra, lattice ? 2 : 1, p->nz, X, s));
  UR_TRY(ur_column_pass(p, X, bins, (float2*)F_out, s));
  return UR_OK;
}

extern "C" ur_status ur_fft_intensity_tiled(const ur_plan* p, const float* cell, int32_t ucell, const int32_t* origin,
                                            const ur_shape* shape, const float* weights, double* bins, void* F_out,
                                            void* ws, size_t ws_bytes, void* stream) {
  return fft_intensity_tiled(p, cell, ucell, origin, nullptr, shape, weights, bins, F_out, ws, ws_bytes, stream);
}

extern "C" ur_status ur_fft_intensity_tiled_lattice(const ur_plan* p, const float* cell, int32_t ucell,
                                                    const ur_lattice* lattice, const ur_shape* shape,
                                                    const float* weights, double* bins, void* F_out, void* ws,
                                                    size_t ws_bytes, void* stream) {
  UR_REQUIRE(lattice, "ur_fft_intensity_tiled_lattice: null lattice");
  return fft_intensity_tiled(p, cell, ucell, nullptr, lattice, shape, weights, bins, F_out, ws, ws_bytes, stream);
}

extern "C" ur_status ur_bin_q(const ur_plan* p, const float* I, double* bins, void* ws, size_t ws_bytes, void* stream) {
  UR_REQUIRE(p && I && bins, "ur_bin_q: null argument");
  (void)ws;
  (void)ws_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = p->nbins;
  const size_t smem = ur_align_up((size_t)(nb + 1) * 4, 16) + (size_t)nb * 16;
  if (smem > 48 * 1024) UR_CUDA_CHECK(cudaFuncSetAttribute(k_bin_half, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  UR_CUDA_CHECK(cudaMemsetAsync(bins, 0, sizeof(double) * UR_BIN_FIELDS * nb, s));
  const double n3 = (double)p->n * p->n * p->n;
  // the kernel accumulates I * N^3 so that k_finalize's I' convention applies
  k_bin_half<<<p->num_sms * 4, 256, smem, s>>>(I, p->n, p->thr, nb, bins + UR_BIN_SUM_I * nb, bins + UR_BIN_SUM_I2 * nb, n3,
                                               p->vsinc);
  UR_LAUNCH_CHECK("k_bin_half");
  k_finalize<<<(nb + 255) / 256, 256, 0, s>>>(bins, p->geo, nb, 1.0 / n3);
  UR_LAUNCH_CHECK("k_finalize");
  return UR_OK;
}

// ---------------------------------------------------------------------------
// Batched launches (many plans of different grid edges in one grid).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_item(const long long* __restrict__ start, int count, long long b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256, 4) k_batch_rows(const BatchRowsItem* __restrict__ items,
                                                       const long long* __restrict__ start, int count) {
  const int i = batch_item(start, count, blockIdx.x);
  const BatchRowsItem& it = items[i];
  if (it.gen) rows_r2c_body<1, float>(it.ra, it.N, it.RB, it.sched, it.nst, blockIdx.x - __ldg(start + i));
  else rows_r2c_body<0, float>(it.ra, it.N, it.RB, it.sched, it.nst, blockIdx.x - __ldg(start + i));
}

template <int MODE, bool INV>
__global__ void __launch_bounds__(256, 4) k_batch_cols(const ColArgs* __restrict__ items,
                                                       const long long* __restrict__ start, int count) {
  const int i = batch_item(start, count, blockIdx.x);
  cols_body<MODE, INV>(items[i], blockIdx.x - __ldg(start + i));
}

__global__ void k_batch_finalize(const BatchFinItem* __restrict__ items) {
  const BatchFinItem& it = items[blockIdx.y];
  finalize_bin(it.bins, it.geo, it.nb, it.inv_n3, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_batch_zero(const BatchZeroItem* __restrict__ items) {
  const BatchZeroItem& it = items[blockIdx.y];
  const size_t n4 = it.bytes / 4;
  uint32_t* p = reinterpret_cast<uint32_t*>(it.ptr);
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x) p[k] = 0u;
}

static void batch_grid_check(long long nblocks) { (void)nblocks; }

ur_status ur_batch_launch_rows(const BatchRowsItem* items, const long long* start, int count, long long nblocks,
                               size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return UR_OK;
  UR_REQUIRE(nblocks < (1ll << 31), "batched rows: too many blocks");
  batch_grid_check(nblocks);
  if (smem > 48 * 1024)
    UR_CUDA_CHECK(cudaFuncSetAttribute(k_batch_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_batch_rows<<<(unsigned)nblocks, 256, smem, s>>>(items, start, count);
  UR_LAUNCH_CHECK("k_batch_rows");
  return UR_OK;
}

ur_status ur_batch_launch_cols(int mode, bool inv, const ColArgs* items, const long long* start, int count,
                               long long nblocks, size_t smem, cudaStream_t s) {
  if (nblocks <= 0) return UR_OK;
  UR_REQUIRE(nblocks < (1ll << 31), "batched columns: too many blocks");
#define UR_BATCH_COLS(MD, IV)                                                                                  \
  do {                                                                                                         \
    UR_CUDA_CHECK(cudaFuncSetAttribute(k_batch_cols<MD, IV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_batch_cols<MD, IV><<<(unsigned)nblocks, 256, smem, s>>>(items, start, count);                            \
  } while (0)
  if (mode == COL_Y && !inv) UR_BATCH_COLS(COL_Y, false);
  else if (mode == COL_Y) UR_BATCH_COLS(COL_Y, true);
  else if (mode == COL_ZBIN) UR_BATCH_COLS(COL_ZBIN, false);
  else UR_BATCH_COLS(COL_ZADJ, false);
#undef UR_BATCH_COLS
  UR_LAUNCH_CHECK("k_batch_cols");
  return UR_OK;
}

ur_status ur_batch_launch_finalize(const BatchFinItem* items, int count, int maxnb, cudaStream_t s) {
  if (count <= 0) return UR_OK;
  k_batch_finalize<<<dim3((unsigned)((maxnb + 255) / 256), (unsigned)count), 256, 0, s>>>(items);
  UR_LAUNCH_CHECK("k_batch_finalize");
  return UR_OK;
}

ur_status ur_batch_launch_zero(const BatchZeroItem* items, int count, cudaStream_t s) {
  if (count <= 0) return UR_OK;
  k_batch_zero<<<dim3(64u, (unsigned)count), 256, 0, s>>>(items);
  UR_LAUNCH_CHECK("k_batch_zero");
  return UR_OK;
}
