// Electron-density generation (Sec. 2.3).
//
// k_density  ED-1: the unit cell repeated with periodic wrap, times the
//            particle mask, written plane by plane (FP32 or FP16).
// k_zoom     ED-2/ED-3: block integration of ED-1 over f^3 blocks, placed
//            in the centre of a zero box (the two orthogonal block steps of
//            the paper are one exact sum here).
#include <math.h>
#include <string.h>

#include <type_traits>

#include "ur_forward.cuh"
#include "ur_density.cuh"

template <typename T>
__device__ __forceinline__ void store2(T* out, float a, float b);
template <>
__device__ __forceinline__ void store2<float>(float* out, float a, float b) {
  *reinterpret_cast<float2*>(out) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void store2<__half>(__half* out, float a, float b) {
  *reinterpret_cast<__half2*>(out) = __halves2half2(__float2half_rn(a), __float2half_rn(b));
}

// grid (ceil(N*N/2 / blockDim), z_count): each thread writes two neighbouring voxels of a row
template <typename T, bool LAT>
__global__ void __launch_bounds__(256) k_density(int N, const float* __restrict__ cell, int U, int ox, int oy, int oz,
                                                 ShapeArgs sh, LatArgs lat, const float* __restrict__ weights,
                                                 int z_begin, T* __restrict__ out, int* __restrict__ nz_range) {
  const int z = z_begin + blockIdx.y;
  const long long pair = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long plane_pairs = (long long)N * N / 2;
  bool nonzero = false;
  if (pair < plane_pairs) {
    const int y = (int)(pair / (N / 2));
    const int x = (int)(pair - (long long)y * (N / 2)) * 2;
    const int cz = (z + oz) % U, cy = (y + oy) % U;
    const float* crow = cell + ((long long)cz * U + cy) * U;
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int xx = x + e;
      const float u = LAT ? lattice_sample(lat, sh, cell, U, xx, y, z) : __ldg(crow + (xx + ox) % U);
      float m;
      if (sh.kind == UR_SHAPE_WEIGHTS) m = __ldg(weights + ((long long)z * N + y) * N + xx);
      else m = mask_at(sh, xx, y, z);
      v[e] = __fmul_rn(u, m);
      // nonzero as stored (an FP16 value may round to zero)
      if (sizeof(T) == 2) v[e] = __half2float(__float2half_rn(v[e]));
    }
    nonzero = (v[0] != 0.f) || (v[1] != 0.f);
    store2<T>(out + ((long long)blockIdx.y * N + y) * N + x, v[0], v[1]);
  }
  if (nz_range) {
    if (__syncthreads_or(nonzero) && threadIdx.x == 0) {
      atomicMin(nz_range, z);
      atomicMax(nz_range + 1, z);
    }
  }
}

static ur_status shape_args(const ur_shape* shape, ShapeArgs* sh) {
  UR_REQUIRE(shape, "ur_build_density: null shape");
  UR_REQUIRE(shape->kind >= UR_SHAPE_SPHERE && shape->kind <= UR_SHAPE_WEIGHTS, "ur_build_density: bad shape kind %d",
             shape->kind);
  *sh = ur_shape_args(shape);
  return UR_OK;
}

static ur_status build_density(int32_t n, const float* cell, int32_t ucell, const int32_t* origin,
                               const ur_lattice* lattice, const ur_shape* shape, const float* weights, int32_t z_begin,
                               int32_t z_count, int32_t out_dtype, void* ed_out, int32_t* nz_range, void* stream) {
  UR_REQUIRE(n >= 2 && n % 2 == 0 && n <= 65536, "ur_build_density: grid edge %d must be even", n);
  UR_REQUIRE(cell && ed_out && ucell >= 1, "ur_build_density: null cell/output or empty cell");
  UR_REQUIRE(z_begin >= 0 && z_count >= 0 && z_begin + z_count <= n, "ur_build_density: planes [%d, %d) outside [0, %d)",
             z_begin, z_begin + z_count, n);
  UR_REQUIRE(out_dtype == UR_F32 || out_dtype == UR_F16, "ur_build_density: out_dtype must be UR_F32 or UR_F16");
  UR_REQUIRE(((uintptr_t)ed_out % 8) == 0, "ur_build_density: ed_out must be 8-byte aligned");
  ShapeArgs sh;
  UR_TRY(shape_args(shape, &sh));
  UR_REQUIRE(sh.kind != UR_SHAPE_WEIGHTS || weights, "ur_build_density: weights required for UR_SHAPE_WEIGHTS");
  int ox = 0, oy = 0, oz = 0;
  if (origin) {
    UR_REQUIRE(origin[0] >= 0 && origin[1] >= 0 && origin[2] >= 0, "ur_build_density: origin must be >= 0");
    ox = origin[0];
    oy = origin[1];
    oz = origin[2];
  }
  const LatArgs lat = ur_lattice_args(lattice);
  if (z_count == 0) return UR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const long long pairs = (long long)n * n / 2;
  dim3 grid((unsigned)((pairs + 255) / 256), (unsigned)z_count);
  ur_timing_begin("density", s);
  if (out_dtype == UR_F32 && !lat.on)
    k_density<float, false><<<grid, 256, 0, s>>>(n, cell, ucell, ox, oy, oz, sh, lat, weights, z_begin, (float*)ed_out,
                                                 nz_range);
  else if (out_dtype == UR_F32)
    k_density<float, true><<<grid, 256, 0, s>>>(n, cell, ucell, ox, oy, oz, sh, lat, weights, z_begin, (float*)ed_out,
                                                nz_range);
  else if (!lat.on)
    k_density<__half, false><<<grid, 256, 0, s>>>(n, cell, ucell, ox, oy, oz, sh, lat, weights, z_begin,
                                                  (__half*)ed_out, nz_range);
  else
    k_density<__half, true><<<grid, 256, 0, s>>>(n, cell, ucell, ox, oy, oz, sh, lat, weights, z_begin,
                                                 (__half*)ed_out, nz_range);
  UR_LAUNCH_CHECK("k_density");
  ur_timing_end(s);
  return UR_OK;
}

extern "C" ur_status ur_build_density(int32_t n, const float* cell, int32_t ucell, const int32_t* origin,
                                      const ur_shape* shape, const float* weights, int32_t z_begin, int32_t z_count,
                                      int32_t out_dtype, void* ed_out, int32_t* nz_range, void* stream) {
  return build_density(n, cell, ucell, origin, nullptr, shape, weights, z_begin, z_count, out_dtype, ed_out, nz_range,
                       stream);
}

extern "C" ur_status ur_build_density_lattice(int32_t n, const float* cell, int32_t ucell, const ur_lattice* lattice,
                                              const ur_shape* shape, const float* weights, int32_t z_begin,
                                              int32_t z_count, int32_t out_dtype, void* ed_out, int32_t* nz_range,
                                              void* stream) {
  UR_REQUIRE(lattice, "ur_build_density_lattice: null lattice");
  return build_density(n, cell, ucell, nullptr, lattice, shape, weights, z_begin, z_count, out_dtype, ed_out, nz_range,
                       stream);
}

// ---------------------------------------------------------------------------
// Zoom-out by block integration
// ---------------------------------------------------------------------------
// Round v = S * 2^-24 (S an integer) to binary16, ties to even.
__device__ __forceinline__ unsigned short half_bits_from_fixed24(long long S) {
  unsigned short sign = 0;
  unsigned long long a;
  if (S < 0) {
    sign = 0x8000;
    a = (unsigned long long)(-S);
  } else {
    a = (unsigned long long)S;
  }
  if (a < 1024ull) return sign | (unsigned short)a;  // subnormal or zero: exact
  int e = 63 - __clzll((long long)a);               // a in [2^e, 2^(e+1)), e >= 10
  const int shift = e - 10;
  unsigned long long q = a >> shift;
  if (shift > 0) {
    const unsigned long long rem = a & ((1ull << shift) - 1);
    const unsigned long long half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    if (q == 2048ull) {
      q = 1024ull;
      ++e;
    }
  }
  const int ex = e - 9;  // biased exponent of q * 2^(e - 10 - 24)
  if (ex >= 31) return sign | 0x7C00;
  return sign | (unsigned short)((ex << 10) | (int)(q - 1024ull));
}

// One block per output row (Z, Y) of the n_out^3 box.
template <typename TS, typename TO>
__global__ void __launch_bounds__(256) k_zoom(const TS* __restrict__ src, int n_src, int f, int n_out,
                                              TO* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Z = blockIdx.x / n_out, Y = blockIdx.x - (blockIdx.x / n_out) * n_out;
  const int m = n_src / f, o = (n_out - m) / 2;
  const int zs = Z - o, ys = Y - o;
  TO* orow = out + ((long long)Z * n_out + Y) * n_out;
  const bool inside = zs >= 0 && zs < m && ys >= 0 && ys < m;
  constexpr bool EXACT = sizeof(TS) == 2;
  using Acc = typename std::conditional<EXACT, unsigned long long, double>::type;
  Acc* acc = reinterpret_cast<Acc*>(smraw);
  if (inside) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) acc[i] = 0;
    __syncthreads();
    for (int x = threadIdx.x; x < n_src; x += blockDim.x) {
      Acc part = 0;
      for (int dz = 0; dz < f; ++dz) {
        for (int dy = 0; dy < f; ++dy) {
          const long long row = ((long long)(f * zs + dz) * n_src + (f * ys + dy)) * n_src;
          if constexpr (EXACT) {
            const float v = __half2float(src[row + x]);
            part += (unsigned long long)__float2ll_rn(v * 16777216.0f);  // v * 2^24, an exact integer
          } else {
            part += (double)src[row + x];
          }
        }
      }
      atomicAdd(acc + x / f, part);
    }
    __syncthreads();
  }
  for (int X = threadIdx.x; X < n_out; X += blockDim.x) {
    const int xs = X - o;
    float vf = 0.f;
    unsigned short hb = 0;
    if (inside && xs >= 0 && xs < m) {
      if constexpr (EXACT) {
        const long long S = (long long)acc[xs];
        hb = half_bits_from_fixed24(S);
        vf = __double2float_rn((double)S * 5.9604644775390625e-08);  // * 2^-24, exact in double
      } else {
        const double d = (double)acc[xs];
        vf = __double2float_rn(d);
        hb = __half_as_ushort(__double2half(d));
      }
    }
    if constexpr (sizeof(TO) == 2) orow[X] = __ushort_as_half(hb);
    else orow[X] = vf;
  }
}

extern "C" ur_status ur_zoom_density(int32_t n_src, int32_t src_dtype, const void* src, int32_t f, int32_t n_out,
                                     int32_t out_dtype, void* out, void* stream) {
  UR_REQUIRE(src && out, "ur_zoom_density: null argument");
  UR_REQUIRE(f >= 1 && n_src >= f && n_src % f == 0, "ur_zoom_density: source edge %d not divisible by factor %d", n_src, f);
  UR_REQUIRE(n_out >= n_src / f, "ur_zoom_density: box %d smaller than the zoomed particle %d", n_out, n_src / f);
  UR_REQUIRE(src_dtype == UR_F32 || src_dtype == UR_F16, "ur_zoom_density: bad source type");
  UR_REQUIRE(out_dtype == UR_F32 || out_dtype == UR_F16, "ur_zoom_density: bad output type");
  UR_REQUIRE(src_dtype == UR_F32 || (long long)f * f * f <= 4096, "ur_zoom_density: FP16 exact sums need f^3 <= 4096");
  cudaStream_t s = (cudaStream_t)stream;
  const int m = n_src / f;
  const size_t smem = (size_t)m * 8;
  UR_REQUIRE(smem <= 200 * 1024, "ur_zoom_density: zoomed row too long");
  const unsigned grid = (unsigned)((long long)n_out * n_out);
#define UR_ZOOM(TS, TO)                                                                                   \
  do {                                                                                                    \
    if (smem > 48 * 1024)                                                                                 \
      UR_CUDA_CHECK(cudaFuncSetAttribute(k_zoom<TS, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_zoom<TS, TO><<<grid, 256, smem, s>>>((const TS*)src, n_src, f, n_out, (TO*)out);                    \
  } while (0)
  ur_timing_begin("zoom", s);
  if (src_dtype == UR_F16 && out_dtype == UR_F16) UR_ZOOM(__half, __half);
  else if (src_dtype == UR_F16) UR_ZOOM(__half, float);
  else if (out_dtype == UR_F16) UR_ZOOM(float, __half);
  else UR_ZOOM(float, float);
#undef UR_ZOOM
  UR_LAUNCH_CHECK("k_zoom");
  ur_timing_end(s);
  return UR_OK;
}
