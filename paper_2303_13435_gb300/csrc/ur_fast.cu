// Power-of-two grid edges (64 <= N <= 4096): compile-time transforms.
//
// A length-L line is held by L/8 threads, eight complex values each
// (thread j holds positions j + q L/8, q = 0..7).  Each Stockham stage is a
// radix-8 butterfly in registers (the last stage radix 4 or 2 when log2 L is
// not a multiple of 3); between stages the values cross shared memory once,
// at padded addresses i + i/16 so that neither the strided writes nor the
// contiguous reads conflict in banks.  After the last stage a thread again
// holds positions j + q L/8, so the first stage can read and the last stage
// can write global memory directly.
//
// Kernels (Sec. 2.4 Eq. 2 split, Sec. 2.5 binning, and the adjoint):
//   k_p2_rows<N, GEN>  rows along x: real-to-complex via an N/2-point
//                      transform; GEN = 1 generates the density of the row
//                      on the fly (Sec. 2.3 tile + mask) instead of reading ED
//   k_p2_cols<N, MODE> columns along y (in place or into another buffer,
//                      forward or inverse) or along z (+ |F|^2 binning, or the
//                      adjoint's scale-and-invert)
//   k_p2_rows_grad<N>  inverse real transform along x + dL/dm, dL/du
#include <math.h>
#include <string.h>

#include "ur_density.cuh"
#include "ur_fast.cuh"

// E = values per thread: 8 (radix-8 stages) or 16 (radix-16 stages, used by the
// column passes of the longest lines, where fewer exchanges per transform and
// more values per barrier pay for the registers).
template <int L, int E = 8>
struct P2 {
  static constexpr int LOG = L == 8 ? 3 : L == 16 ? 4 : L == 32 ? 5 : L == 64 ? 6 : L == 128 ? 7 : L == 256 ? 8
                                                                                           : L == 512 ? 9 : L == 1024 ? 10
                                                                                           : L == 2048 ? 11 : 12;
  static constexpr int LE = E == 16 ? 4 : 3;  // log2 E
  static constexpr int T = L / E;
  static constexpr int NFULL = LOG / LE;
  static constexpr int REM = LOG % LE;
  static constexpr int NST = NFULL + (REM ? 1 : 0);
  static constexpr int PITCH = L + L / 16;
  static_assert(E == 8 || E == 16, "8 or 16 values per thread");
};

__device__ __forceinline__ int p2pad(int i) { return i + (i >> 4); }

constexpr int ipowe(int e, int s) { return s == 0 ? 1 : e * ipowe(e, s - 1); }

// Offset (float2) of stage S >= 1 in the stage twiddle table of an L-point transform:
// the stages before S are radix E, with E^s rows of E slots each.
template <int E>
constexpr int p2_stage_off(int S) { return S <= 1 ? 0 : p2_stage_off<E>(S - 1) + E * ipowe(E, S - 1); }

// Butterflies of stage S.  Thread j runs E/R butterflies b = j + i L/E; the
// inputs of butterfly i are v[i + (E/R) r], r < R; k = b mod NS; the twiddles
// exp(-+2 pi i r k/(NS R)), r = 1 .. R-1, are row k of the stage's block of the
// stage table (plan-built in float64, stored float32; E slots per row), read as
// 16-byte pairs.
template <int L, int E, int R, int NS, int S, bool INV>
__device__ __forceinline__ void p2_butterflies(float2 (&v)[E], int j, const float2* __restrict__ stw) {
  constexpr int T = L / E, NB = E / R;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = j + i * T;
    const int k = b & (NS - 1);
    float2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = v[i + NB * r];
    if constexpr (NS > 1) {
      const float4* row = reinterpret_cast<const float4*>(stw + p2_stage_off<E>(S) + k * E);
      float2 w[R];
#pragma unroll
      for (int h = 0; h < R / 2; ++h) {
        const float4 t = __ldg(row + h);
        w[2 * h] = make_float2(t.x, t.y);
        w[2 * h + 1] = make_float2(t.z, t.w);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) a[r] = twmul<INV>(a[r], w[r]);
    }
    dft<R, INV>(a);
#pragma unroll
    for (int r = 0; r < R; ++r) v[i + NB * r] = a[r];
  }
}

// Barrier between the writers and readers of a line: the whole block, or only
// the warp when every thread of the line sits in one warp (L/E <= 32).
template <bool WS>
__device__ __forceinline__ void p2_sync(unsigned wmask) {
  if constexpr (WS) __syncwarp(wmask);
  else __syncthreads();
}

// lanes of the warp that hold the line of this thread (T <= 32 threads per line)
template <int T>
__device__ __forceinline__ unsigned p2_line_lanes() {
  if constexpr (T >= 32) return 0xffffffffu;
  else return ((1u << T) - 1u) << ((threadIdx.x & 31) & ~(T - 1));
}

// Stage outputs to shared memory at (b - k) R + k + r NS, then reload as j + q L/E.
template <int L, int E, int R, int NS, bool WS>
__device__ __forceinline__ void p2_exchange(float2 (&v)[E], int j, float2* line, unsigned wmask) {
  constexpr int T = L / E, NB = E / R;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = j + i * T;
    const int k = b & (NS - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) line[p2pad((b - k) * R + k + r * NS)] = v[i + NB * r];
  }
  p2_sync<WS>(wmask);
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = line[p2pad(j + q * T)];
  p2_sync<WS>(wmask);
}

template <int L, int E, bool INV, bool WS, int S>
struct P2Run {
  __device__ static __forceinline__ void run(float2 (&v)[E], int j, float2* line, const float2* __restrict__ stw,
                                             unsigned wmask) {
    constexpr int NST = P2<L, E>::NST, NFULL = P2<L, E>::NFULL, REM = P2<L, E>::REM;
    if constexpr (S < NST) {
      constexpr int R = (S < NFULL) ? E : (1 << REM);
      constexpr int NS = ipowe(E, S);
      p2_butterflies<L, E, R, NS, S, INV>(v, j, stw);
      if constexpr (S + 1 < NST) p2_exchange<L, E, R, NS, WS>(v, j, line, wmask);
      P2Run<L, E, INV, WS, S + 1>::run(v, j, line, stw, wmask);
    }
  }
};

// Whole line transform.  WS = false: every thread of the block must call it
// (block barriers); WS = true: the L/E threads of a line share a warp and all
// of them (the lanes in wmask) must call it.  stw: the stage twiddle table of
// the L-point transform for E values per thread.
template <int L, bool INV, bool WS = false, int E = 8>
__device__ __forceinline__ void p2_fft(float2 (&v)[E], int j, float2* line, const float2* __restrict__ stw,
                                       unsigned wmask = 0xffffffffu) {
  P2Run<L, E, INV, WS, 0>::run(v, j, line, stw, wmask);
}

// ---------------------------------------------------------------------------
// Rows: real-to-complex along x (pass 1a), optionally generating the density.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float2 ld_pair(const T* p);
template <>
__device__ __forceinline__ float2 ld_pair<float>(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
template <>
__device__ __forceinline__ float2 ld_pair<__half>(const __half* p) {
  return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
}

template <int N, int GEN, typename TED>
__global__ void __launch_bounds__(512, 3) k_p2_rows(RowArgs a) {
  constexpr int M = N / 2, H = M + 1, T = M / 8, RB = 512 / T, PITCH = P2<M>::PITCH;
  // a row of up to 256 complex values is one warp (or part of one): warp barriers only
  constexpr bool WS = T <= 32;
  __shared__ __align__(16) float2 sm[RB * PITCH];
  const int t = threadIdx.x / T, j = threadIdx.x - (threadIdx.x / T) * T;
  const long long r = (long long)blockIdx.x * RB + t;
  const bool valid = r < a.nrows;
  const unsigned wmask = p2_line_lanes<T>();
  float2* line = sm + t * PITCH;
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = make_float2(0.f, 0.f);
  if (GEN) {
    const int p = (int)(r / N), y = (int)(r - (long long)p * N);
    const int z = a.z0 + p;
    RowMask rm;
    rm.init(a.sh, y, z);
    const int U = a.ucell;
    const float* wrow = a.weights ? a.weights + ((long long)z * N + y) * N : nullptr;
    if constexpr (WS) {
      // rows outside the sphere: not written at all when the y pass knows to skip them
      // (the condition is uniform over the row's lanes, which only sync among themselves)
      if (a.skip_empty && valid && !wrow && rm.empty()) return;
    }
    // rows the mask excludes entirely are zero (cell values are finite)
    if (valid && (wrow || !rm.empty())) {
      if constexpr (GEN == 2) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int x = 2 * (j + q * T);
          float m0, m1;
          if (wrow) {
            const float2 mw = __ldg(reinterpret_cast<const float2*>(wrow + x));
            m0 = mw.x;
            m1 = mw.y;
          } else {
            m0 = rm.at(x);
            m1 = rm.at(x + 1);
          }
          const float u0 = m0 != 0.f ? lattice_sample(a.lat, a.sh, a.cell, U, x, y, z) : 0.f;
          const float u1 = m1 != 0.f ? lattice_sample(a.lat, a.sh, a.cell, U, x + 1, y, z) : 0.f;
          v[q] = make_float2(__fmul_rn(u0, m0), __fmul_rn(u1, m1));
        }
      } else {
        const float* crow = a.cell + ((long long)a.fu.mod(z + a.oz) * U + a.fu.mod(y + a.oy)) * U;
        // cell column of x = 2 (j + q T): one modulo per thread, then steps of 2T mod U
        const int cstep = a.fu.mod(2 * T);
        int c0 = a.fu.mod(2 * j + a.ox);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int x = 2 * (j + q * T);
          float m0, m1;
          if (wrow) {
            const float2 mw = __ldg(reinterpret_cast<const float2*>(wrow + x));
            m0 = mw.x;
            m1 = mw.y;
          } else {
            m0 = rm.at(x);
            m1 = rm.at(x + 1);
          }
          const float u0 = __ldg(crow + c0), u1 = __ldg(crow + (c0 + 1 == U ? 0 : c0 + 1));
          c0 += cstep;
          if (c0 >= U) c0 -= U;
          v[q] = make_float2(__fmul_rn(u0, m0), __fmul_rn(u1, m1));
        }
      }
    }
  } else if (valid) {
    const TED* row = reinterpret_cast<const TED*>(a.ed) + r * N;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = ld_pair<TED>(row + 2 * (j + q * T));
  }
  // a row whose values are all zero transforms to zero: skip its butterflies
  bool zero_row = false;
  if constexpr (WS) {
    bool nz = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) nz |= (v[q].x != 0.f) || (v[q].y != 0.f);
    zero_row = (__ballot_sync(wmask, nz) & wmask) == 0u;
  }
  if (!zero_row) p2_fft<M, false, WS>(v, j, line, a.stw, wmask);
  // split step: X[k] = (Z[k] + conj Z[M-k])/2 - i W_N^k (Z[k] - conj Z[M-k])/2
  if constexpr (WS) {
    // Z[M - k], k = j + qT, is register 7 - q of lane T - j of the same row (j >= 1);
    // lane j = 0 holds its own partners: Z[M - qT] = its register 8 - q, and Z[0]
    const int src = ((threadIdx.x & 31) & ~(T - 1)) | ((T - j) & (T - 1));
    float2* X = a.X + (valid ? r : 0) * H;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float2 zm = make_float2(__shfl_sync(wmask, v[7 - q].x, src), __shfl_sync(wmask, v[7 - q].y, src));
      if (j == 0) zm = v[(8 - q) & 7];
      if (!valid) continue;
      const int k = j + q * T;
      if (zero_row) {
        X[k] = make_float2(0.f, 0.f);
        continue;
      }
      const float2 zk = v[q], zc = cconj(zm);
      const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
      const float2 d = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
      const float2 o = make_float2(d.y, -d.x);
      X[k] = cadd(e, cmul(__ldg(a.tw + k), o));
    }
    if (valid && j == 0) {  // k = M: Z[M] = Z[0]
      const float2 zk = v[0], zc = cconj(v[0]);
      const float2 d = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
      X[M] = cadd(make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y)),
                  cmul(__ldg(a.tw + M), make_float2(d.y, -d.x)));
    }
    return;
  }
  if (!zero_row) {
#pragma unroll
    for (int q = 0; q < 8; ++q) line[p2pad(j + q * T)] = v[q];
  }
  p2_sync<WS>(wmask);
  if (valid) {
    float2* X = a.X + r * H;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      int k = j + q * T;
      if (q == 8) {
        if (j != 0) break;
        k = M;
      }
      if (zero_row) {
        X[k] = make_float2(0.f, 0.f);
        continue;
      }
      const float2 zk = line[p2pad(k == M ? 0 : k)];
      const float2 zc = cconj(line[p2pad(k == 0 ? 0 : M - k)]);
      const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
      const float2 d = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
      const float2 o = make_float2(d.y, -d.x);
      X[k] = cadd(e, cmul(__ldg(a.tw + k), o));
    }
  }
}

// ---------------------------------------------------------------------------
// Columns.  Block = TX columns x L/E threads; thread (j, c), c fastest, so a
// warp reads whole row segments of TX consecutive columns.
// ---------------------------------------------------------------------------
enum { P2_Y_FWD = 0, P2_Y_INV = 1, P2_Z_BIN = 2, P2_Z_ADJ = 3 };

// E: values per thread (ur_fast_col_e); threads per column block: 512, or 1024
// for N >= 2048 so that a block still spans at least two columns (16-byte row
// segments) of the half spectrum.  MINB: resident blocks per SM the register
// budget is cut for (the z pass with binning fits in 32 registers: four blocks
// of 512 threads; 16 values per thread take 64)
template <int N, int MODE = P2_Y_FWD>
struct ColCfg {
  static constexpr int E = UR_FAST_COL_E(N);
  static constexpr int THREADS = N >= 2048 ? 1024 : 512;
  static constexpr int TX = THREADS / (N / E);
  static constexpr int MINB = E == 16 ? 65536 / (64 * THREADS) : N >= 2048 ? 2 : MODE == P2_Z_BIN ? 4 : 3;
};

template <int N, int MODE>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, (ColCfg<N, MODE>::MINB)) k_p2_cols(ColArgs a) {
  // column pitch = 2 (mod 16) float2: the TX columns a warp touches fall on different banks
  constexpr int E = ColCfg<N>::E;
  constexpr int T = N / E, TX = ColCfg<N>::TX, PITCH = P2<N>::PITCH + 2, H = N / 2 + 1, M = N / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_blo, s_bhi;
  float2* buf = reinterpret_cast<float2*>(smraw);
  constexpr size_t BUF_BYTES = ((size_t)TX * PITCH * sizeof(float2) + 15) / 16 * 16;
  int32_t* thr = reinterpret_cast<int32_t*>(smraw + BUF_BYTES);
  float* hs = reinterpret_cast<float*>(smraw + BUF_BYTES + ur_align_up_dev((size_t)(a.nbins + 1) * 4, 16));
  float* hs2 = hs + a.nbins;
  int16_t* crs = reinterpret_cast<int16_t*>(reinterpret_cast<unsigned char*>(hs) +
                                            ur_align_up_dev((size_t)a.nbins * 8, 16));  // 16-byte aligned
  float* Kb = reinterpret_cast<float*>(crs);  // forward binning: the block's cache of the bin shifts
  const int c = threadIdx.x % TX, j = threadIdx.x / TX;
  const int col0 = blockIdx.x * TX;
  const int col = col0 + c;
  const bool valid = col < a.ncols;
  const bool binning = (MODE == P2_Z_BIN || MODE == P2_Z_ADJ) && a.nbins > 0;
  // column position of the spectrum (z passes): kx, ky
  int kx = 0, ky = 0;
  {
    const int o = col / H;
    kx = col - o * H;
    ky = o < M ? o : o - N;
  }
  const int c2 = kx * kx + ky * ky;
  // z passes: the bin thresholds go to shared memory.  The adjoint, which needs the bin
  // of every element, also stages the coarse rank table and its per-bin scales there (no
  // gathers from global memory per element).  The forward binning needs only a few bins
  // per column: the bins a column can reach lie between those of k^2 = c2 and c2 + M^2,
  // read here from the full k^2 -> bin table and used after the column loads.
  int lo_bin = 0, hi_bin = 0;
  if (MODE == P2_Z_BIN && binning) {
    if (threadIdx.x == 0) {
      s_blo = 0x7fffffff;
      s_bhi = -1;
    }
    if (j == 0 && valid) {
      const int nb = a.nbins, t0 = __ldg(a.thr), tn = __ldg(a.thr + nb);
      const int s_lo = c2, s_hi = c2 + M * M;
      lo_bin = s_lo < t0 ? 0 : s_lo >= tn ? nb - 1 : __ldg(a.lut + s_lo);
      hi_bin = s_hi < t0 ? 0 : s_hi >= tn ? nb - 1 : __ldg(a.lut + s_hi);
    }
  }
  // z passes: columns whose k^2 = kx^2 + ky^2 already lies at or beyond the closing
  // threshold reach no bin at any kz.  A block made only of such columns has nothing to
  // bin (forward, when F is not written) or only zero scales (adjoint: its output is
  // zero), so it skips the loads and the transforms.
  const bool skip_mode = (MODE == P2_Z_BIN && binning && !a.fout) || (MODE == P2_Z_ADJ && binning);
  if (skip_mode) {
    // every thread votes for its own column (columns past the end count as beyond); in the
    // forward the vote's barrier also publishes the range reset above
    const bool beyond = __syncthreads_and(!valid || c2 >= __ldg(a.thr + a.nbins));
    if (beyond) {  // uniform over the block
      // adjoint: the output columns are zero; unless the caller reads them as zeros
      // without loading (k2_zero), write them
      if (MODE == P2_Z_ADJ && valid && a.k2_zero == 0x7fffffff) {
        const long long dbase = (long long)(col / H) * a.Ad + (col - (col / H) * H);
#pragma unroll
        for (int q = 0; q < E; ++q) a.dst[dbase + (long long)(j + q * T) * a.Sd] = make_float2(0.f, 0.f);
      }
      return;
    }
  }
  if (MODE == P2_Z_ADJ && binning) {  // staged by the blocks that transform
    for (int i = threadIdx.x; i <= a.nbins; i += blockDim.x) thr[i] = __ldg(a.thr + i);
    for (int i = threadIdx.x; i < UR_COARSE_ENTRIES / 8; i += blockDim.x)
      reinterpret_cast<uint4*>(crs)[i] = __ldg(reinterpret_cast<const uint4*>(a.crs) + i);
    for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) hs[i] = __ldg(a.sigma + i);
  }
  const long long sbase = (long long)(col / H) * a.A + (col - (col / H) * H);
  float2 v[E];
  if (MODE == P2_Y_FWD && a.row_skip) {
    // forward y pass over a generated sphere: rows y outside the particle in plane z are
    // zero and were not written by the row pass
    const float2* src = a.src + (valid ? sbase + (long long)j * a.S : 0);
    const long long step = (long long)T * a.S;
    const int z = a.gen_z0 + col / H;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int y = j + q * T;
      v[q] = (valid && !sphere_row_empty(a.sh, y, z)) ? __ldg(src + q * step) : make_float2(0.f, 0.f);
    }
  } else if (MODE == P2_Y_INV && a.k2_zero != 0x7fffffff) {
    // adjoint y pass: elements with kx^2 + ky^2 >= k2_zero are zero (the z pass left them
    // unwritten) and are not read
    const float2* src = a.src + (valid ? sbase + (long long)j * a.S : 0);
    const long long step = (long long)T * a.S;
    const int kx2 = kx * kx;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int li = j + q * T, kyy = li < M ? li : li - N;
      v[q] = (valid && kx2 + kyy * kyy < a.k2_zero) ? __ldg(src + q * step) : make_float2(0.f, 0.f);
    }
  } else if (a.zoff == 0 && a.nload == N) {  // whole column present (y passes, F given)
    const float2* src = a.src + (valid ? sbase + (long long)j * a.S : 0);
    const long long step = (long long)T * a.S;
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = __ldg(src + q * step);
  } else {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int li = j + q * T - a.zoff;
      v[q] = (valid && li >= 0 && li < a.nload) ? __ldg(a.src + sbase + (long long)li * a.S) : make_float2(0.f, 0.f);
    }
  }
  // forward z pass: the thresholds go to shared memory after the column loads are issued, so
  // that the two latencies overlap (the adjoint stages its tables before its loads: staged
  // after them, the loaded values stay live across the staging and spill at 40 registers)
  if (MODE == P2_Z_BIN && binning) {
    for (int i = threadIdx.x; i <= a.nbins; i += blockDim.x) thr[i] = __ldg(a.thr + i);
  }
  float2* line = buf + c * PITCH;
  if (binning && (MODE == P2_Z_ADJ || !skip_mode)) __syncthreads();  // tables (and the range reset) visible
  if (MODE == P2_Z_BIN && binning && j == 0 && valid) {
    // the block's histogram range [s_blo, s_bhi] is zeroed after the transform, whose
    // barriers order it after these updates
    atomicMin(&s_blo, lo_bin);
    atomicMax(&s_bhi, hi_bin);
  }
  if (MODE == P2_Y_FWD || MODE == P2_Y_INV) {
    p2_fft<N, MODE == P2_Y_INV, false, E>(v, j, line, a.stw);
    if (valid) {
      const long long dbase = (long long)(col / H) * a.Ad + (col - (col / H) * H);
#pragma unroll
      for (int q = 0; q < E; ++q) a.dst[dbase + (long long)(j + q * T) * a.Sd] = v[q];
    }
  } else if (MODE == P2_Z_BIN) {
    p2_fft<N, false, false, E>(v, j, line, a.stw);
    if (a.fout && valid) {
#pragma unroll
      for (int q = 0; q < E; ++q) a.fout[(long long)(j + q * T) * N * H + col] = cscale(v[q], a.fscale);
    }
    if (binning) {
      // task = (column, chunk of CH consecutive |kz| = m); at most one task per thread.
      // The bin of the chunk's first m comes from the k^2 table (its load is issued
      // before the barrier below); after that the bin only moves forward, when
      // s = c2 + m^2 (updated by 2m + 1) reaches the next threshold, so the loop over
      // the chunk compares, accumulates a run of equal bins and flushes it on a change.
      constexpr int CH = (H + T - 1) / T;
      constexpr int NCH = (H + CH - 1) / CH;
      static_assert(TX * NCH <= ColCfg<N>::THREADS, "one binning task per thread");
      const int nb = a.nbins;
      const int tc = threadIdx.x % TX, ch = threadIdx.x / TX;
      const int gcol = col0 + tc;
      const bool has = ch < NCH && gcol < a.ncols;
      int cc2 = 0, m0 = 0, bcur = 0;
      float w = 0.f, csc = a.iscale;  // csc: I scale of the column (times its voxel-sinc factor)
      if (has) {
        const int o2 = gcol / H, kx2 = gcol - o2 * H, ky2 = o2 < M ? o2 : o2 - N;
        cc2 = kx2 * kx2 + ky2 * ky2;
        w = (kx2 == 0 || kx2 == M) ? 1.f : 2.f;
        if (a.vs) csc = a.iscale * (__ldg(a.vs + kx2) * __ldg(a.vs + (ky2 < 0 ? -ky2 : ky2)));
        m0 = ch * CH;
        const int s0 = cc2 + m0 * m0;
        bcur = s0 < thr[0] ? -1 : s0 >= thr[nb] ? nb : __ldg(a.lut + s0);
      }
      for (int i = s_blo + (int)threadIdx.x; i <= s_bhi; i += blockDim.x) {
        hs[i] = 0.f;
        hs2[i] = 0.f;
        // the shifts already published for the block's bins, fetched together up front (a
        // fetch inside the walk would stall it); unset ones are NaN and published on first use
        const unsigned long long g = __ldcg(a.gK + i);
        Kb[i] = g ? __uint_as_float((unsigned)(g & 0xffffffffull)) : __int_as_float(0x7fc00000);
      }
      // natural order in shared memory
#pragma unroll
      for (int q = 0; q < E; ++q) line[p2pad(j + q * T)] = v[q];
      __syncthreads();
      if (has) {
        const float2* ln = buf + tc * PITCH;
        int b = bcur;
        int tnext = b < nb ? thr[b + 1] : 0x7fffffff;
        int s = cc2 + m0 * m0;
        // shifted run sums: sum (I - K) and sum (I - K)^2 with the bin's shift K (ur_bin_shift)
        float sI = 0.f, sI2 = 0.f, K = 0.f;
        bool fresh = true;
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int mm = m0 + u;
          if (mm <= M) {
            if (s >= tnext) {
              if (b >= 0) {
                atomicAdd(hs + b, w * sI);
                atomicAdd(hs2 + b, w * sI2);
              }
              sI = 0.f;
              sI2 = 0.f;
              fresh = true;
              do {
                ++b;
                tnext = b < nb ? thr[b + 1] : 0x7fffffff;
              } while (s >= tnext);
            }
            if (b >= 0 && b < nb) {
              const float sc = a.vs ? csc * __ldg(a.vs + mm) : csc;
              const float2 f1 = ln[p2pad(mm)];
              const float i1 = (f1.x * f1.x + f1.y * f1.y) * sc;
              if (fresh) {
                K = ur_bin_shift(Kb, a.gK, b, i1);
                fresh = false;
              }
              const float d1 = i1 - K;
              sI += d1;
              sI2 = fmaf(d1, d1, sI2);
              if (mm != 0 && mm != M) {
                const float2 f2 = ln[p2pad(N - mm)];
                const float d2 = (f2.x * f2.x + f2.y * f2.y) * sc - K;
                sI += d2;
                sI2 = fmaf(d2, d2, sI2);
              }
            }
            s += 2 * mm + 1;
          }
        }
        if (b >= 0 && b < nb) {
          atomicAdd(hs + b, w * sI);
          atomicAdd(hs2 + b, w * sI2);
        }
      }
      __syncthreads();
      for (int i = s_blo + (int)threadIdx.x; i <= s_bhi; i += blockDim.x) {
        if (hs[i] != 0.f) atomicAdd(a.gsum + i, (double)hs[i]);
        if (hs2[i] != 0.f) atomicAdd(a.gsum2 + i, (double)hs2[i]);
      }
    }
  } else {  // P2_Z_ADJ
    if (!a.skip_fwd) p2_fft<N, false, false, E>(v, j, line, a.stw);
    // scale of element kz: sigma of the bin of k^2 = c2 + m^2, m = |signed kz|
    const int nb = a.nbins;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int kz = j + q * T;
      const int m = kz <= M ? kz : N - kz;
      const int b = bin_rank(crs, a.crs_shift, thr, nb, c2 + m * m);
      v[q] = cscale(v[q], (b >= 0 && b < nb) ? hs[b] : 0.f);
    }
    p2_fft<N, true, false, E>(v, j, line, a.stw);
    if (valid) {
      const long long dbase = (long long)(col / H) * a.Ad + (col - (col / H) * H);
      if (a.out_cnt > 0) {  // a slab of output planes
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int zo = j + q * T - a.out_lo;
          if (zo >= 0 && zo < a.out_cnt) a.dst[dbase + (long long)zo * a.Sd] = v[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < E; ++q) a.dst[dbase + (long long)(j + q * T) * a.Sd] = v[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint rows: inverse real transform along x, then dL/dm and dL/du.
// Block = RB rows (z, y) that share the cell row (cz, cy): y = yf + U t.
//   Z[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k]) conj(W_N^k),
//   z = IFFT_{N/2}(Z),  (g(2m), g(2m+1)) = (Re z[m], Im z[m]).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(512, 3) k_p2_rows_grad(GradArgs a) {
  constexpr int M = N / 2, H = M + 1, T = M / 8, PITCH = P2<M>::PITCH + 1;
  constexpr bool WS = T <= 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int RB = a.rb;
  float2* sm = reinterpret_cast<float2*>(smraw);
  float* acc = reinterpret_cast<float*>(smraw + ur_align_up_dev((size_t)RB * PITCH * sizeof(float2), 16));
  const int U = a.ucell;
  const int t = threadIdx.x / T, j = threadIdx.x - (threadIdx.x / T) * T;
  const unsigned wmask = p2_line_lanes<T>();
  const int cy = blockIdx.y;
  const int z = a.z0 + blockIdx.z;
  const int cz = (z + a.oz) % U;
  const int yt = cy - a.oy + U;  // (cy - oy) mod U with 0 <= oy < U
  const int yf = yt >= U ? yt - U : yt;
  const int y = yf + U * (blockIdx.x * RB + t);
  const bool valid = y < N;
  for (int i = threadIdx.x; i < U; i += blockDim.x) acc[i] = 0.f;
  float2* line = sm + t * PITCH;
  const float2* Yrow = a.Y + ((long long)(z - a.ybase_z) * N + (valid ? y : 0)) * H;
  // all nine loads of the row (k = j + q T, and k = M) are issued together
  float2 ld[9];
#pragma unroll
  for (int q = 0; q < 8; ++q) ld[q] = valid ? __ldg(Yrow + j + q * T) : make_float2(0.f, 0.f);
  ld[8] = (valid && j == 0) ? __ldg(Yrow + M) : make_float2(0.f, 0.f);
  float2 v[8];
  if constexpr (WS) {
    // X[M - k], k = j + qT, is load 7 - q of lane T - j of the same row (j >= 1); lane
    // j = 0 holds its own partners: X[M - qT] = its load 8 - q (X[M] for q = 0)
    const int src = ((threadIdx.x & 31) & ~(T - 1)) | ((T - j) & (T - 1));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = j + q * T;
      float2 xb = make_float2(__shfl_sync(wmask, ld[7 - q].x, src), __shfl_sync(wmask, ld[7 - q].y, src));
      if (j == 0) xb = ld[8 - q];
      const float2 xa = ld[q];
      const float2 w = __ldg(a.tw + k);
      const float2 e = cadd(xa, cconj(xb));
      const float2 d = csub(xa, cconj(xb));
      const float2 o = make_float2(d.x * w.x + d.y * w.y, d.y * w.x - d.x * w.y);
      v[q] = make_float2(e.x - o.y, e.y + o.x);
    }
    __syncthreads();  // orders the zeroing of acc before any accumulation
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) line[p2pad(j + q * T)] = ld[q];
    if (j == 0) line[p2pad(M)] = ld[8];
    __syncthreads();  // also orders the zeroing of acc before any accumulation
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = j + q * T;
      const float2 xa = line[p2pad(k)], xb = line[p2pad(M - k)];
      const float2 w = __ldg(a.tw + k);
      const float2 e = cadd(xa, cconj(xb));
      const float2 d = csub(xa, cconj(xb));
      const float2 o = make_float2(d.x * w.x + d.y * w.y, d.y * w.x - d.x * w.y);
      v[q] = make_float2(e.x - o.y, e.y + o.x);
    }
    __syncthreads();  // the transform's first exchange reuses the lines
  }
  p2_fft<M, true, WS>(v, j, line, a.stw, wmask);
  const float* crow = a.cell + ((long long)cz * U + cy) * U;
  RowMask rm;
  rm.init(a.sh, valid ? y : 0, z);
  const float* wrow = a.weights ? a.weights + ((long long)z * N + (valid ? y : 0)) * N : nullptr;
  if (valid) {
    float* drow = a.dl_dmask ? a.dl_dmask + ((long long)(z - a.mbase_z) * N + y) * N : nullptr;
    // rows the mask excludes entirely add nothing to dL/du
    const bool mzero = !wrow && rm.empty();
    // cell columns of x = 2 (j + q T): one modulo, then steps of 2T mod U; when U divides
    // 2T they are the same for every q and the dL/du sums stay in two registers
    const int cstep = a.cstep;
    int c0 = 2 * j + a.ox;  // reduced below: 0 <= ox < U
    while (c0 >= U) c0 -= U;
    if (cstep == 0) {
      const int c1 = c0 + 1 == U ? 0 : c0 + 1;
      const float u0 = __ldg(crow + c0), u1 = __ldg(crow + c1);
      float r0 = 0.f, r1 = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int x = 2 * (j + q * T);
        const float g0 = v[q].x * a.inv_n3, g1 = v[q].y * a.inv_n3;
        if (drow) *reinterpret_cast<float2*>(drow + x) = make_float2(g0 * u0, g1 * u1);
        if (!mzero) {
          float m0, m1;
          if (wrow) {
            const float2 mw = __ldg(reinterpret_cast<const float2*>(wrow + x));
            m0 = mw.x;
            m1 = mw.y;
          } else {
            m0 = rm.at(x);
            m1 = rm.at(x + 1);
          }
          r0 += g0 * m0;
          r1 += g1 * m1;
        }
      }
      if (r0 != 0.f) atomicAdd(acc + c0, r0);
      if (r1 != 0.f) atomicAdd(acc + c1, r1);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int x = 2 * (j + q * T);
        const float g0 = v[q].x * a.inv_n3, g1 = v[q].y * a.inv_n3;
        const int c1 = c0 + 1 == U ? 0 : c0 + 1;
        if (drow) *reinterpret_cast<float2*>(drow + x) = make_float2(g0 * __ldg(crow + c0), g1 * __ldg(crow + c1));
        if (!mzero) {
          float m0, m1;
          if (wrow) {
            const float2 mw = __ldg(reinterpret_cast<const float2*>(wrow + x));
            m0 = mw.x;
            m1 = mw.y;
          } else {
            m0 = rm.at(x);
            m1 = rm.at(x + 1);
          }
          if (m0 != 0.f) atomicAdd(acc + c0, g0 * m0);
          if (m1 != 0.f) atomicAdd(acc + c1, g1 * m1);
        }
        c0 += cstep;
        if (c0 >= U) c0 -= U;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < U; i += blockDim.x)
    if (acc[i] != 0.f) atomicAdd(a.dl_dcell + ((long long)cz * U + cy) * U + i, acc[i]);
}

// ---------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------
bool ur_fast_supported(int n) {
  return n == 64 || n == 128 || n == 256 || n == 512 || n == 1024 || n == 2048 || n == 4096;
}

template <int N>
static size_t cols_smem(int nbins, int mode) {
  constexpr int TX = ColCfg<N>::TX, PITCH = P2<N>::PITCH + 2;
  return ur_align_up((size_t)TX * PITCH * sizeof(float2), 16) + ur_align_up((size_t)(nbins + 1) * 4, 16) +
         ur_align_up((size_t)nbins * 8, 16) + (mode == P2_Z_ADJ ? (size_t)UR_COARSE_ENTRIES * 2 : 0) +
         (mode == P2_Z_BIN ? (size_t)nbins * 4 : 0);
}

template <int N>
static ur_status launch_cols_n(int mode, const ColArgs& a, cudaStream_t s) {
  constexpr int TX = ColCfg<N>::TX;
  const size_t smem = cols_smem<N>(a.nbins, mode);
  const int grid = (int)((a.ncols + TX - 1) / TX);
  if (grid <= 0) return UR_OK;
#define UR_P2_LAUNCH(MD)                                                                                   \
  do {                                                                                                     \
    UR_CUDA_CHECK(cudaFuncSetAttribute(k_p2_cols<N, MD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_p2_cols<N, MD><<<grid, ColCfg<N>::THREADS, smem, s>>>(a);                                                           \
  } while (0)
  switch (mode) {
    case P2_Y_FWD: UR_P2_LAUNCH(P2_Y_FWD); break;
    case P2_Y_INV: UR_P2_LAUNCH(P2_Y_INV); break;
    case P2_Z_BIN: UR_P2_LAUNCH(P2_Z_BIN); break;
    default: UR_P2_LAUNCH(P2_Z_ADJ); break;
  }
#undef UR_P2_LAUNCH
  UR_LAUNCH_CHECK("k_p2_cols");
  return UR_OK;
}

ur_status ur_fast_cols(int n, int mode, const ColArgs& a, cudaStream_t s) {
  switch (n) {
    case 64: return launch_cols_n<64>(mode, a, s);
    case 128: return launch_cols_n<128>(mode, a, s);
    case 256: return launch_cols_n<256>(mode, a, s);
    case 512: return launch_cols_n<512>(mode, a, s);
    case 1024: return launch_cols_n<1024>(mode, a, s);
    case 2048: return launch_cols_n<2048>(mode, a, s);
    case 4096: return launch_cols_n<4096>(mode, a, s);
  }
  ur_set_error("ur_fast_cols: unsupported size %d", n);
  return UR_ERR_UNSUPPORTED;
}

template <int N>
static ur_status launch_rows_n(const RowArgs& a, int gen, int ed_f16, cudaStream_t s) {
  constexpr int M = N / 2, T = M / 8, RB = 512 / T;
  const int grid = (int)((a.nrows + RB - 1) / RB);
  if (grid <= 0) return UR_OK;
  if (gen == 2) k_p2_rows<N, 2, float><<<grid, 512, 0, s>>>(a);
  else if (gen) k_p2_rows<N, 1, float><<<grid, 512, 0, s>>>(a);
  else if (ed_f16) k_p2_rows<N, 0, __half><<<grid, 512, 0, s>>>(a);
  else k_p2_rows<N, 0, float><<<grid, 512, 0, s>>>(a);
  UR_LAUNCH_CHECK("k_p2_rows");
  return UR_OK;
}

ur_status ur_fast_rows(int n, const RowArgs& a, int gen, int ed_f16, cudaStream_t s) {
  switch (n) {
    case 64: return launch_rows_n<64>(a, gen, ed_f16, s);
    case 128: return launch_rows_n<128>(a, gen, ed_f16, s);
    case 256: return launch_rows_n<256>(a, gen, ed_f16, s);
    case 512: return launch_rows_n<512>(a, gen, ed_f16, s);
    case 1024: return launch_rows_n<1024>(a, gen, ed_f16, s);
    case 2048: return launch_rows_n<2048>(a, gen, ed_f16, s);
    case 4096: return launch_rows_n<4096>(a, gen, ed_f16, s);
  }
  ur_set_error("ur_fast_rows: unsupported size %d", n);
  return UR_ERR_UNSUPPORTED;
}

template <int N>
static ur_status launch_grad_n(GradArgs a, int nplanes, cudaStream_t s) {
  constexpr int M = N / 2, T = M / 8, PITCH = P2<M>::PITCH + 1;
  const int U = a.ucell;
  const int rows_per_group = (N + U - 1) / U;
  int rb = 512 / T;
  if (rb > rows_per_group) rb = rows_per_group;
  a.rb = rb;
  a.cstep = (2 * T) % U;
  const size_t smem = ur_align_up((size_t)rb * PITCH * sizeof(float2), 16) + (size_t)U * sizeof(float);
  UR_REQUIRE(smem <= 200 * 1024, "adjoint rows: cell edge %d too large", U);
  if (smem > 48 * 1024) UR_CUDA_CHECK(cudaFuncSetAttribute(k_p2_rows_grad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)((rows_per_group + rb - 1) / rb), (unsigned)U, (unsigned)nplanes);
  if (nplanes <= 0) return UR_OK;
  k_p2_rows_grad<N><<<grid, rb * T, smem, s>>>(a);
  UR_LAUNCH_CHECK("k_p2_rows_grad");
  return UR_OK;
}

ur_status ur_fast_rows_grad(int n, const GradArgs& a, int nplanes, cudaStream_t s) {
  switch (n) {
    case 64: return launch_grad_n<64>(a, nplanes, s);
    case 128: return launch_grad_n<128>(a, nplanes, s);
    case 256: return launch_grad_n<256>(a, nplanes, s);
    case 512: return launch_grad_n<512>(a, nplanes, s);
    case 1024: return launch_grad_n<1024>(a, nplanes, s);
    case 2048: return launch_grad_n<2048>(a, nplanes, s);
    case 4096: return launch_grad_n<4096>(a, nplanes, s);
  }
  ur_set_error("ur_fast_rows_grad: unsupported size %d", n);
  return UR_ERR_UNSUPPORTED;
}
