// Ewald-sphere detector image (Sec. 2.5, first paragraph): for anisotropic
// samples, the 2D pattern a practical experiment records is the 3D intensity
// read on the Ewald sphere, a shell whose thickness the wavelength
// distribution sets.
//
// One thread per detector pixel.  Pixel (ix, iy) of a flat detector normal to
// the beam at distance L sees the direction s of ((ix - bx) p, (iy - by) p, L);
// for each of nl wavelengths lambda_l = lambda0 (1 + b ((l + 1/2)/nl - 1/2)) the
// sample-frame scattering vector is q = R^T (2 pi / lambda_l)(s - z_hat), i.e.
// the fractional frequency k = (N dx / lambda_l) R^T (s - z_hat).  The
// intensity |F|^2 at k is the trilinear interpolation over the 8 neighbouring
// grid frequencies, read from the half spectrum through F(-k) = conj F(k).  A
// sample counts when every neighbour lies in [-N/2, N/2 - 1] on every axis;
// the pixel is the mean over its counted samples (NaN if none).
// s - z_hat is formed as (x, y, -(x^2 + y^2)/(L + r)) / r, which keeps its
// small z component accurate in float32.
#include <math.h>

#include "ur_forward.cuh"

struct EwaldArgs {
  int nx, ny, nl, N, H;
  float bx, by, pix, L;
  float kscale[16];  // N dx / lambda_l
  float r[9];
};

__device__ __forceinline__ float ewald_I(const float2* __restrict__ F, int N, int H, int kx, int ky, int kz) {
  if (kx < 0) {
    kx = -kx;
    ky = -ky;
    kz = -kz;
  }
  const int iy = ky < 0 ? ky + N : ky, iz = kz < 0 ? kz + N : kz;
  const float2 f = __ldg(F + ((long long)iz * N + iy) * H + kx);
  return f.x * f.x + f.y * f.y;
}

__global__ void k_ewald(EwaldArgs a, const float2* __restrict__ F, float* __restrict__ img) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  if (ix >= a.nx) return;
  const float x = ((float)ix - a.bx) * a.pix, y = ((float)iy - a.by) * a.pix;
  const float rho2 = x * x + y * y;
  const float r = sqrtf(rho2 + a.L * a.L);
  const float d[3] = {x / r, y / r, -rho2 / ((a.L + r) * r)};
  // R^T d
  float e[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) e[c] = a.r[c] * d[0] + a.r[3 + c] * d[1] + a.r[6 + c] * d[2];
  const int half = a.N / 2;
  float sum = 0.f;
  int cnt = 0;
  for (int l = 0; l < a.nl; ++l) {
    const float kf[3] = {a.kscale[l] * e[0], a.kscale[l] * e[1], a.kscale[l] * e[2]};
    int i0[3];
    float f[3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float fl = floorf(kf[c]);
      i0[c] = (int)fl;
      f[c] = kf[c] - fl;
      ok = ok && i0[c] >= -half && i0[c] + 1 <= half - 1;
    }
    if (!ok) continue;
    float v = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) * (dz ? f[2] : 1.f - f[2]);
          v += w * ewald_I(F, a.N, a.H, i0[0] + dx, i0[1] + dy, i0[2] + dz);
        }
    sum += v;
    ++cnt;
  }
  img[(long long)iy * a.nx + ix] = cnt > 0 ? sum / (float)cnt : __int_as_float(0x7fc00000);
}

extern "C" ur_status ur_ewald_image(const ur_plan* p, const void* F_half, const ur_detector* det, float* image,
                                    void* stream) {
  UR_REQUIRE(p && F_half && det && image, "ur_ewald_image: null argument");
  UR_REQUIRE(det->nx >= 1 && det->ny >= 1 && det->ny <= 65535, "ur_ewald_image: bad detector size %d x %d", det->nx,
             det->ny);
  UR_REQUIRE(det->nlambda >= 1 && det->nlambda <= 16, "ur_ewald_image: nlambda %d outside [1, 16]", det->nlambda);
  UR_REQUIRE(det->pixel_m > 0 && det->distance_m > 0 && det->wavelength_nm > 0 && det->bandwidth >= 0 &&
                 det->bandwidth < 2,
             "ur_ewald_image: pixel, distance and wavelength must be positive, bandwidth in [0, 2)");
  UR_REQUIRE(((uintptr_t)F_half % 8) == 0, "ur_ewald_image: F must be 8-byte aligned");
  EwaldArgs a;
  a.nx = det->nx;
  a.ny = det->ny;
  a.nl = det->nlambda;
  a.N = p->n;
  a.H = p->H;
  a.bx = (float)det->beam_x;
  a.by = (float)det->beam_y;
  a.pix = (float)det->pixel_m;
  a.L = (float)det->distance_m;
  for (int l = 0; l < 16; ++l) a.kscale[l] = 0.f;
  for (int l = 0; l < det->nlambda; ++l) {
    const double lam = det->wavelength_nm * (1.0 + det->bandwidth * ((l + 0.5) / det->nlambda - 0.5));
    a.kscale[l] = (float)((double)p->n * p->dx / lam);
  }
  for (int i = 0; i < 9; ++i) a.r[i] = det->rot[i];
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid((unsigned)((det->nx + 127) / 128), (unsigned)det->ny);
  k_ewald<<<grid, 128, 0, s>>>(a, (const float2*)F_half, image);
  UR_LAUNCH_CHECK("k_ewald");
  return UR_OK;
}
