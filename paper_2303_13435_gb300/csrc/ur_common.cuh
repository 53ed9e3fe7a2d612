// Internal definitions shared by the CUDA translation units of libur.
//
// Complex arithmetic, the small DFT butterflies, the shared-memory Stockham
// FFT engine, integer bin lookup, and the plan structure.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "ur.h"

// ---------------------------------------------------------------------------
// Host error reporting
// ---------------------------------------------------------------------------
void ur_set_error(const char* fmt, ...);
ur_status ur_fault_point(const char* site);  // host-side fault injection (UR_FAULT=<site>:<n>)

#define UR_CUDA_CHECK(call)                                                                  \
  do {                                                                                       \
    cudaError_t ur_e_ = (call);                                                              \
    if (ur_e_ != cudaSuccess) {                                                              \
      ur_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(ur_e_), __FILE__, __LINE__); \
      return UR_ERR_CUDA;                                                                    \
    }                                                                                        \
  } while (0)

#define UR_LAUNCH_CHECK(name)                                                                \
  do {                                                                                       \
    cudaError_t ur_e_ = cudaGetLastError();                                                  \
    if (ur_e_ != cudaSuccess) {                                                              \
      ur_set_error("launch of %s failed: %s", name, cudaGetErrorString(ur_e_));             \
      return UR_ERR_CUDA;                                                                    \
    }                                                                                        \
  } while (0)

#define UR_REQUIRE(cond, ...)                                                                \
  do {                                                                                       \
    if (!(cond)) {                                                                           \
      ur_set_error(__VA_ARGS__);                                                             \
      return UR_ERR_INVALID;                                                                 \
    }                                                                                        \
  } while (0)

#define UR_TRY(expr)                      \
  do {                                    \
    ur_status ur_s_ = (expr);             \
    if (ur_s_ != UR_OK) return ur_s_;     \
  } while (0)

// ---------------------------------------------------------------------------
// Division by a run-time constant: q = (umulhi(x, m) + x) >> s with
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1 (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994).
// Exact for 0 <= x < 2^31 and 1 <= d < 2^31.
// ---------------------------------------------------------------------------
struct FastDiv {
  uint32_t d, m, s;
  __host__ __device__ FastDiv() : d(1), m(1), s(0) {}
  __host__ __device__ explicit FastDiv(uint32_t dd) : d(dd) {
    uint32_t sh = 0;
    while ((1ull << sh) < dd) ++sh;
    s = sh;
    m = (uint32_t)(((1ull << 32) * ((1ull << sh) - dd)) / dd + 1);
  }
  __host__ __device__ __forceinline__ uint32_t div(uint32_t x) const {
#ifdef __CUDA_ARCH__
    uint32_t hi = __umulhi(x, m);
#else
    uint32_t hi = (uint32_t)(((uint64_t)x * m) >> 32);
#endif
    return (hi + x) >> s;
  }
  __host__ __device__ __forceinline__ uint32_t mod(uint32_t x) const { return x - div(x) * d; }
};

// ---------------------------------------------------------------------------
// Complex helpers (float2 = re, im); host-callable so the library can check its
// butterflies against a direct DFT without a GPU.
#define UR_HD __host__ __device__
// ---------------------------------------------------------------------------
UR_HD __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
UR_HD __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
UR_HD __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
UR_HD __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
UR_HD __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (-i) for the forward direction, a * (+i) for the inverse
template <bool INV>
UR_HD __forceinline__ float2 mul_ni(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// Twiddle load through the read-only path.  The asm is volatile so that the
// compiler does not hoist the (loop-invariant) loads of every stage out of a
// kernel's outer loop and keep them all in registers.
__device__ __forceinline__ float2 ld_twiddle(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
// a * W where W is the forward twiddle (inverse: conj(W))
template <bool INV>
UR_HD __forceinline__ float2 twmul(float2 a, float2 w) {
  return INV ? make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y) : cmul(a, w);
}

// ---------------------------------------------------------------------------
// Small DFTs in registers.  Forward: y_p = sum_m a_m exp(-2 pi i m p / R);
// inverse: the conjugate kernel (no scaling).
// ---------------------------------------------------------------------------
template <bool INV>
UR_HD __forceinline__ void dft2(float2& a0, float2& a1) {
  float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <bool INV>
UR_HD __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  float2 t2 = cadd(a1, a3), t3 = mul_ni<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <bool INV>
UR_HD __forceinline__ void dft8(float2* a) {
  // even/odd split into two 4-point DFTs, then W8^k combination
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float r = 0.70710678118654752f;
  // o1 *= W8^1, o2 *= W8^2, o3 *= W8^3
  if (!INV) {
    o1 = make_float2((o1.x + o1.y) * r, (o1.y - o1.x) * r);
    o2 = make_float2(o2.y, -o2.x);
    o3 = make_float2((o3.y - o3.x) * r, -(o3.x + o3.y) * r);
  } else {
    o1 = make_float2((o1.x - o1.y) * r, (o1.x + o1.y) * r);
    o2 = make_float2(-o2.y, o2.x);
    o3 = make_float2(-(o3.x + o3.y) * r, (o3.x - o3.y) * r);
  }
  a[0] = cadd(e0, o0);
  a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1);
  a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2);
  a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3);
  a[7] = csub(e3, o3);
}

// Odd prime R in {3, 5, 7}: pair a_m with a_{R-m}; y_p = t_p -/+ i u_p.
template <int R>
struct OddConst;
template <>
struct OddConst<3> {
  __host__ __device__ static constexpr float c(int q) { return -0.5f; }
  __host__ __device__ static constexpr float s(int q) { return q == 1 ? 0.86602540378443865f : -0.86602540378443865f; }
};
template <>
struct OddConst<5> {
  __host__ __device__ static constexpr float c(int q) {
    return (q == 1 || q == 4) ? 0.30901699437494742f : -0.80901699437494742f;
  }
  __host__ __device__ static constexpr float s(int q) {
    return q == 1 ? 0.95105651629515357f : q == 2 ? 0.58778525229247313f : q == 3 ? -0.58778525229247313f
                                                                                  : -0.95105651629515357f;
  }
};
template <>
struct OddConst<7> {
  __host__ __device__ static constexpr float c(int q) {
    return (q == 1 || q == 6) ? 0.62348980185873353f : (q == 2 || q == 5) ? -0.22252093395631440f
                                                                           : -0.90096886790241913f;
  }
  __host__ __device__ static constexpr float s(int q) {
    return q == 1 ? 0.78183148246802981f : q == 2 ? 0.97492791218182361f : q == 3 ? 0.43388373911755812f
           : q == 4 ? -0.43388373911755812f : q == 5 ? -0.97492791218182361f : -0.78183148246802981f;
  }
};

template <int R, bool INV>
UR_HD __forceinline__ void dft_odd(float2* a) {
  constexpr int h = (R - 1) / 2;
  float2 b[h], d[h];
#pragma unroll
  for (int m = 1; m <= h; ++m) {
    b[m - 1] = cadd(a[m], a[R - m]);
    d[m - 1] = csub(a[m], a[R - m]);
  }
  float2 y0 = a[0];
#pragma unroll
  for (int m = 0; m < h; ++m) y0 = cadd(y0, b[m]);
  float2 y[R];
  y[0] = y0;
#pragma unroll
  for (int p = 1; p <= h; ++p) {
    float2 t = a[0];
    float2 u = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 1; m <= h; ++m) {
      const int q = (m * p) % R;
      const float cc = OddConst<R>::c(q), ss = OddConst<R>::s(q);
      t.x = fmaf(cc, b[m - 1].x, t.x);
      t.y = fmaf(cc, b[m - 1].y, t.y);
      u.x = fmaf(ss, d[m - 1].x, u.x);
      u.y = fmaf(ss, d[m - 1].y, u.y);
    }
    // forward: y_p = t - i u, y_{R-p} = t + i u
    float2 iu = make_float2(-u.y, u.x);
    if (!INV) {
      y[p] = csub(t, iu);
      y[R - p] = cadd(t, iu);
    } else {
      y[p] = cadd(t, iu);
      y[R - p] = csub(t, iu);
    }
  }
#pragma unroll
  for (int p = 0; p < R; ++p) a[p] = y[p];
}

// exp(-2 pi i m / 32) from the first octant of cos(2 pi m / 32) (float64 literals)
UR_HD constexpr float ur_cos32(int m) {
  constexpr float c[9] = {1.0f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                          0.70710678118654752f, 0.55557023301960218f, 0.38268343236508977f, 0.19509032201612825f, 0.0f};
  m &= 31;
  return m <= 8 ? c[m] : m <= 16 ? -c[16 - m] : m <= 24 ? -c[m - 16] : c[32 - m];
}
UR_HD constexpr float ur_w32_re(int m) { return ur_cos32(m); }
UR_HD constexpr float ur_w32_im(int m) { return -ur_cos32(m - 8); }  // -sin(2 pi m / 32)

// exp(-2 pi i m / L), m < L, for the inner twiddles of composite radices L that
// do not divide 32: cos and sin from their Taylor series, summed in double at
// compile time on the argument reduced to [-pi, pi], then rounded to float.
UR_HD constexpr double ur_ct_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 30; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
UR_HD constexpr double ur_ct_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 30; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
template <int L>
struct UrTw {
  float re[L], im[L];
  UR_HD constexpr UrTw() : re(), im() {
    constexpr double pi = 3.14159265358979323846;
    for (int m = 0; m < L; ++m) {
      double x = 2.0 * pi * (double)m / (double)L;
      if (x > pi) x -= 2.0 * pi;
      re[m] = (float)ur_ct_cos(x);
      im[m] = (float)(-ur_ct_sin(x));
    }
  }
};

// L = R1 R2 point DFT from R1- and R2-point DFTs (n = R2 n1 + n2, k = k1 + R1 k2):
//   X[k1 + R1 k2] = sum_n2 W_R2^(n2 k2) [W_L^(n2 k1) sum_n1 a[R2 n1 + n2] W_R1^(n1 k1)]
template <int R, bool INV>
UR_HD __forceinline__ void dft(float2* a);

template <int R1, int R2, bool INV>
UR_HD __forceinline__ void dft_split(float2* a) {
  constexpr int L = R1 * R2;
  float2 y[L];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    float2 t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = a[R2 * n1 + n2];
    dft<R1, INV>(t);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      if constexpr (32 % L == 0) {
        const int m = (n2 * k1 * (32 / L)) & 31;
        y[n2 * R1 + k1] = (n2 * k1 == 0) ? t[k1] : twmul<INV>(t[k1], make_float2(ur_w32_re(m), ur_w32_im(m)));
      } else {
        constexpr UrTw<L> W{};
        const int m = (n2 * k1) % L;
        y[n2 * R1 + k1] = (n2 * k1 == 0) ? t[k1] : twmul<INV>(t[k1], make_float2(W.re[m], W.im[m]));
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
    dft<R2, INV>(t);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = t[k2];
  }
}

template <int R, bool INV>
UR_HD __forceinline__ void dft(float2* a) {
  if constexpr (R == 2) {
    dft2<INV>(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(a[0], a[1], a[2], a[3]);
  } else if constexpr (R == 8) {
    dft8<INV>(a);
  } else if constexpr (R == 16) {
    dft_split<4, 4, INV>(a);
  } else if constexpr (R == 32) {
    dft_split<4, 8, INV>(a);
  } else if constexpr (R == 6) {
    dft_split<2, 3, INV>(a);
  } else if constexpr (R == 9) {
    dft_split<3, 3, INV>(a);
  } else if constexpr (R == 10) {
    dft_split<2, 5, INV>(a);
  } else {
    dft_odd<R, INV>(a);
  }
}

// ---------------------------------------------------------------------------
// Radix schedule of a length-L FFT that reads its twiddles from a table of
// length n_tab (exp(-2 pi i t / n_tab), generated in float64 on the host).
// Stage st has radix R, butterflies per line nb = L/R, and Ns = product of the
// radices of the earlier stages.
// ---------------------------------------------------------------------------
#define UR_MAX_STAGES 14
// Radices of the shared-memory engine, in the order their stages run (each radix
// has its own loop in fft_lines; a schedule lists its stages in this order).
// (Composites of 12 and more points spilled registers at 64 per thread.)
#define UR_NRADIX 9
static constexpr int ur_radix_order[UR_NRADIX] = {8, 4, 2, 6, 10, 9, 3, 5, 7};
struct StageInfo {
  int R, nb, Ns, tstep;  // tstep = n_tab / (Ns * R)
  FastDiv div_nb, div_ns;
};
struct Sched {
  int L, nst;
  StageInfo st[UR_MAX_STAGES];
};

bool ur_make_sched(int L, int n_tab, Sched* out);  // host; false if L is not {2,3,5,7}-smooth

// One Stockham autosort stage, in place in shared memory (pitch between
// lines), all threads of the block participating.  Each thread first loads
// every input of its butterflies into registers, the block synchronises, and
// then it writes the outputs, so reads and writes of the stage never race.
//   input  of butterfly j (line l): x[l][j + r nb], r = 0..R-1
//   twiddle exp(-2 pi i r k / (Ns R)), k = j mod Ns
//   output y[l][(j - k) R + k + r Ns]
template <int R, bool INV, int EMAX>
__device__ __forceinline__ void fft_stage(float2* __restrict__ buf, int pitch, int lines, const StageInfo& si,
                                          const float2* __restrict__ tw) {
  constexpr int BMAX = (EMAX + R - 1) / R;
  const int nb = si.nb;
  const int total = lines * nb;
  float2 v[BMAX][R];
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int w = threadIdx.x + b * blockDim.x;
    if (w < total) {
      const int line = (int)si.div_nb.div((uint32_t)w);
      const int j = w - line * nb;
      const float2* src = buf + line * pitch + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = src[r * nb];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int w = threadIdx.x + b * blockDim.x;
    if (w < total) {
      const int line = (int)si.div_nb.div((uint32_t)w);
      const int j = w - line * nb;
      const int k = (int)si.div_ns.mod((uint32_t)j);
      if (si.Ns > 1 && k > 0) {
        const int step = k * si.tstep;
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = twmul<INV>(v[b][r], ld_twiddle(tw + r * step));
      }
      dft<R, INV>(v[b]);
      float2* dst = buf + line * pitch + (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * si.Ns] = v[b][r];
    }
  }
  __syncthreads();
}

// FFT of `lines` lines held in shared memory (pitch apart), in place, with the
// stage table `st` (nst stages, device memory).  Requires lines * L <= EMAX *
// blockDim.x.  Every thread of the block must call it.
// The stages of one radix run in their own loop (schedules list radices in
// the order of ur_radix_order): a single loop with a switch over the radix
// makes the compiler keep the register arrays of every case live at once.
template <int R, bool INV, int EMAX>
__device__ __forceinline__ int fft_stages_of(float2* buf, int pitch, int lines, const StageInfo* st, int nst,
                                             const float2* __restrict__ tw, int i) {
  while (i < nst) {  // nst: one past the last stage to run
    const StageInfo si = st[i];  // shared memory (fft_lines): a broadcast read per stage
    if (si.R != R) break;
    fft_stage<R, INV, EMAX>(buf, pitch, lines, si, tw);
    ++i;
  }
  return i;
}

// The schedule is copied to shared memory once per call: reading it from
// global memory at every stage put an L2 round trip in front of each stage.
template <bool INV, int EMAX>
__device__ __forceinline__ void fft_lines(float2* buf, int pitch, int lines, const StageInfo* __restrict__ st, int nst,
                          const float2* __restrict__ tw) {
  static_assert(sizeof(StageInfo) % 4 == 0, "StageInfo is copied as 32-bit words");
  constexpr int W = (int)(sizeof(StageInfo) / 4);
  __shared__ __align__(16) uint32_t s_raw[UR_MAX_STAGES * W];  // raw words: StageInfo has constructors
  const StageInfo* s_st = reinterpret_cast<const StageInfo*>(s_raw);
  __syncthreads();  // an earlier call of this kernel may still read s_raw
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(st);
    for (int w = threadIdx.x; w < nst * W; w += blockDim.x) s_raw[w] = __ldg(src + w);
  }
  __syncthreads();
  int i = 0;
  i = fft_stages_of<8, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<4, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<2, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<6, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<10, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<9, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<3, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<5, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
  i = fft_stages_of<7, INV, EMAX>(buf, pitch, lines, s_st, nst, tw, i);
}

// First stage (Ns = 1, no twiddles) with inputs from `ld(line, i)` instead of shared
// memory, and last stage (k = j, outputs at j + r Ns) handing its outputs to
// `st(line, i, v)`.  Their butterflies are mapped line-fastest (w = j lines + line), so
// consecutive threads take the same position of consecutive lines: a tile of columns is
// read and written in row segments.
template <int R, bool INV, int EMAX, bool LF, class Ld>
__device__ __forceinline__ void fft_first_stage(float2* __restrict__ buf, int pitch, int lines, const FastDiv& dl,
                                                const StageInfo& si, Ld ld) {
  constexpr int BMAX = (EMAX + R - 1) / R;
  const int nb = si.nb;
  const int total = lines * nb;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int w = threadIdx.x + b * blockDim.x;
    if (w < total) {
      int j, line;
      if constexpr (LF) {
        j = (int)dl.div((uint32_t)w);
        line = w - j * lines;
      } else {
        line = (int)si.div_nb.div((uint32_t)w);
        j = w - line * nb;
      }
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = ld(line, j + r * nb);
      dft<R, INV>(v);
      float2* dst = buf + line * pitch + j * R;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r] = v[r];
    }
  }
  __syncthreads();
}

template <int R, bool INV, int EMAX, bool LF, class St>
__device__ __forceinline__ void fft_last_stage(const float2* __restrict__ buf, int pitch, int lines,
                                               const FastDiv& dl, const StageInfo& si,
                                               const float2* __restrict__ tw, St st) {
  constexpr int BMAX = (EMAX + R - 1) / R;
  const int nb = si.nb;
  const int total = lines * nb;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int w = threadIdx.x + b * blockDim.x;
    if (w < total) {
      int j, line;
      if constexpr (LF) {
        j = (int)dl.div((uint32_t)w);
        line = w - j * lines;
      } else {
        line = (int)si.div_nb.div((uint32_t)w);
        j = w - line * nb;
      }
      const float2* src = buf + line * pitch + j;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src[r * nb];
      if (j > 0) {  // last stage: Ns = nb, so k = j
        const int step = j * si.tstep;
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twmul<INV>(v[r], ld_twiddle(tw + r * step));
      }
      dft<R, INV>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) st(line, j + r * nb, v[r]);
    }
  }
}

template <bool INV, int EMAX, bool LF, class Ld>
__device__ __forceinline__ void fft_first_any(float2* buf, int pitch, int lines, const FastDiv& dl,
                                              const StageInfo& si, Ld ld) {
  switch (si.R) {
    case 8: fft_first_stage<8, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 4: fft_first_stage<4, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 2: fft_first_stage<2, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 6: fft_first_stage<6, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 10: fft_first_stage<10, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 9: fft_first_stage<9, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 3: fft_first_stage<3, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    case 5: fft_first_stage<5, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
    default: fft_first_stage<7, INV, EMAX, LF>(buf, pitch, lines, dl, si, ld); break;
  }
}

template <bool INV, int EMAX, bool LF, class St>
__device__ __forceinline__ void fft_last_any(const float2* buf, int pitch, int lines, const FastDiv& dl,
                                             const StageInfo& si, const float2* tw, St st) {
  switch (si.R) {
    case 8: fft_last_stage<8, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 4: fft_last_stage<4, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 2: fft_last_stage<2, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 6: fft_last_stage<6, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 10: fft_last_stage<10, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 9: fft_last_stage<9, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 3: fft_last_stage<3, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    case 5: fft_last_stage<5, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
    default: fft_last_stage<7, INV, EMAX, LF>(buf, pitch, lines, dl, si, tw, st); break;
  }
}

// FFT of `lines` lines.  With LOAD the first stage reads global memory through `ld`
// (otherwise the lines are in shared memory already); with STORE the last stage writes
// global memory through `st` (otherwise the result stays in shared memory, as with
// fft_lines).  LF: the two stages map butterflies line-fastest (tiles of columns, read
// in row segments) or position-fastest (rows, read along the row).  Needs nst >= 2.
// Every thread of the block must call it; with STORE the caller synchronises before it
// reuses buf.
template <bool INV, int EMAX, bool LOAD, bool STORE, bool LF, class Ld, class St>
__device__ __forceinline__ void fft_lines_io(float2* buf, int pitch, int lines, const StageInfo* __restrict__ st,
                                             int nst, const float2* __restrict__ tw, Ld ld, St stf) {
  constexpr int W = (int)(sizeof(StageInfo) / 4);
  __shared__ __align__(16) uint32_t s_raw[UR_MAX_STAGES * W];
  const StageInfo* s_st = reinterpret_cast<const StageInfo*>(s_raw);
  __syncthreads();  // an earlier call of this kernel may still read s_raw or buf
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(st);
    for (int w = threadIdx.x; w < nst * W; w += blockDim.x) s_raw[w] = __ldg(src + w);
  }
  __syncthreads();
  const FastDiv dl((uint32_t)lines);
  if constexpr (LOAD) fft_first_any<INV, EMAX, LF>(buf, pitch, lines, dl, s_st[0], ld);
  const int iend = STORE ? nst - 1 : nst;
  int i = LOAD ? 1 : 0;
  i = fft_stages_of<8, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<4, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<2, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<6, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<10, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<9, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<3, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<5, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  i = fft_stages_of<7, INV, EMAX>(buf, pitch, lines, s_st, iend, tw, i);
  if constexpr (STORE) fft_last_any<INV, EMAX, LF>(buf, pitch, lines, dl, s_st[nst - 1], tw, stf);
}

// ---------------------------------------------------------------------------
// Bin lookup on integer k^2: bin j holds s in [t_j, t_j+1); -1 / B outside.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bin_search(const int32_t* __restrict__ thr, int nb, int s) {
  // largest j in [0, nb] with thr[j] <= s, or -1
  int lo = 0, hi = nb + 1;  // answer + 1 in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (thr[mid] <= s) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// Rank of k^2 = s among the bin thresholds, r(s) = max{j in [0, nb] : thr[j] <= s}
// (-1 below thr[0]); s lies in bin r when 0 <= r < nb.  crs holds r at multiples of
// 2^shift, so the rank of s is reached from crs[s >> shift] by stepping over the few
// thresholds inside that block.  The two tables are small (6 KB and 4 (nb+1) bytes),
// so a kernel that needs the bin of every element keeps them in shared memory.
#define UR_COARSE_ENTRIES 3072
__device__ __forceinline__ int bin_rank(const int16_t* crs, int shift, const int32_t* thr, int nb, int s) {
  int b = crs[s >> shift];
  while (b < nb && thr[b + 1] <= s) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// Shifted bin sums.  The binning kernels of the power-of-two path sum I - K_j and
// (I - K_j)^2 per bin, with one shift K_j per bin for the whole call: the first value
// any block meets in the bin, published once in a 64-bit slot (0 = unset, else
// (1 << 32) | float bits).  A block keeps the shifts it has seen in shared memory (NaN =
// not yet fetched).  With K_j a value of the bin, the sums do not cancel when the
// spread is small, so mean = K + S_d/n and M2 = Q_d - S_d^2/n stay accurate (Chan et
// al.'s shifted-data form of the variance).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ur_bin_shift(float* Kb, unsigned long long* gK, int b, float v) {
  float k = Kb[b];
  if (k != k) {
    // a plain L2 read first: only the first blocks to reach a bin contend on the CAS
    unsigned long long cur = __ldcg(gK + b);
    if (cur == 0ull) {
      const unsigned long long mine = (1ull << 32) | (unsigned long long)__float_as_uint(v);
      cur = atomicCAS(gK + b, 0ull, mine);
      if (cur == 0ull) cur = mine;
    }
    k = __uint_as_float((unsigned)(cur & 0xffffffffull));
    Kb[b] = k;  // every writer stores the same published value
  }
  return k;
}

// bins field 5 holds the shift slots while the sums accumulate (see ur_bin_shift)
__host__ __device__ inline unsigned long long* ur_shift_slots(double* bins, int nb) {
  return reinterpret_cast<unsigned long long*>(bins + UR_BIN_SEM * nb);
}

// Final statistics of bin j from shifted sums S_d (field 1) and Q_d (field 2) in I' = N^3 I
// units, the shift slot (field 5) and the plan's count and sum |Q|.
__device__ __forceinline__ void ur_finalize_shifted(double* __restrict__ bins, const double* __restrict__ geo, int nb,
                                                    double inv_n3, int j) {
  const double n = geo[j];
  const unsigned long long slot = reinterpret_cast<const unsigned long long*>(bins + UR_BIN_SEM * nb)[j];
  const double K = slot ? (double)__uint_as_float((unsigned)(slot & 0xffffffffull)) : 0.0;
  const double sd = bins[UR_BIN_SUM_I * nb + j], qd = bins[UR_BIN_SUM_I2 * nb + j];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double mean = nan, sem = nan, sI = 0.0, sI2 = 0.0;
  if (n > 0) {
    const double mu = K + sd / n;
    double m2 = qd - sd * (sd / n);
    if (m2 < 0) m2 = 0;
    mean = mu * inv_n3;
    const double m2i = m2 * (inv_n3 * inv_n3);
    sI = n * mean;
    sI2 = m2i + n * mean * mean;
    if (n > 1) sem = sqrt(m2i / (n * (n - 1.0)));
  }
  bins[UR_BIN_COUNT * nb + j] = n;
  bins[UR_BIN_SUM_I * nb + j] = sI;
  bins[UR_BIN_SUM_I2 * nb + j] = sI2;
  bins[UR_BIN_SUM_Q * nb + j] = geo[nb + j];
  bins[UR_BIN_MEAN * nb + j] = mean;
  bins[UR_BIN_SEM * nb + j] = sem;
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct ur_plan {
  int n, M, H;       // grid edge, N/2, N/2+1
  double dx, dq;
  int ed_dtype, z0, nz, nbins;
  int device, num_sms;
  float2* tw;        // device [n]
  float2* stw;       // power-of-two path: stage twiddles of the N-point and (at stw_m_off) the N/2-point transforms
  int stw_m_off;
  int32_t* thr;      // device [nbins+1]
  int16_t* binlut;     // device [3 (N/2)^2 + 1]: bin of k^2 = s, -1 outside every bin
  int16_t* bincoarse;  // device [UR_COARSE_ENTRIES]: bin_rank of s = i << coarse_shift
  int coarse_shift;    // smallest shift with (3 (N/2)^2 >> shift) < UR_COARSE_ENTRIES
  int64_t* thr_host; // host   [nbins+1]
  double* geo;       // device [2][nbins]: count, sum |Q|
  Sched sched_n, sched_m;       // host copies
  StageInfo* d_sched;           // device: [0, UR_MAX_STAGES) length N, then length N/2
  // launch configuration
  int row_threads, row_rb;        // forward/inverse row kernels: rows per block
  int col_threads, col_tx;        // column kernels: columns per block
  int zbin_grid;                  // persistent blocks of the binned column pass
  size_t row_smem, col_smem, colbin_smem;
  // workspace layout (bytes)
  size_t ws_inter;   // nz * N * H complex64
  size_t ws_inv;     // N * N * H complex64
  size_t ws_sigma;   // nbins floats (+pad)
  size_t ws_slab;    // one host-staging slab
  int slab_planes;
  int adj_slab_planes;  // output planes per slab of the out-of-core adjoint (ur_backward_slabs)
  // power-of-two path
  int fast;          // 1: compile-time kernels (N a power of two in [64, 1024])
  int chunk_planes;  // planes per chunk of the plane pass / adjoint y and row passes (n: one launch each)
  size_t ws_chunk;   // adjoint chunk buffer (0 when chunk_planes = n: y-inverse in place)
  float* vsinc;       // device [N/2+1] sinc^2(pi m/N) when the voxel-sinc correction is on, else NULL
  // TMA z-column kernel (N = 256, 512; NULL otherwise), used when zc_enabled
  int zc_enabled;
  float2* zc_tw;      // device [N/16][16]: W_N^(t k1)
  int32_t* zc_tiles;  // device: tiles of 16 spectrum columns with a column below the closing threshold
  int zc_ntiles;
};

// kernels launched from host code in other translation units
ur_status ur_launch_geometry(ur_plan* p, cudaStream_t s);
// TMA z-column kernels (ur_zcol.cu)
ur_status ur_zcol_prepare(ur_plan* p);
bool ur_zcol_supported(const ur_plan* p);
ur_status ur_zcol_forward(const ur_plan* p, const float2* X, double* bins, float2* F_out, float iscale, float fscale,
                          cudaStream_t s);
ur_status ur_deverr_take(void);

static inline size_t ur_align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// planes per dL/dm staging sub-slab of the out-of-core adjoint (at most 64, at most a slab)
static inline int ur_adj_dm_planes(const ur_plan* p) { return p->adj_slab_planes < 64 ? p->adj_slab_planes : 64; }
