// Particle-mask predicate and unit-cell lookup shared by the density kernel,
// the fused density + transform row pass and the adjoint row pass (Sec. 2.3).
#pragma once

#include <string.h>

#include "ur_common.cuh"

struct ShapeArgs {
  int kind;
  float cx, cy, cz, s;
  float r[9];
};

// Mask value at voxel (x, y, z): every product and sum rounded separately
// (no contraction), in the order of the ur_build_density contract.
__device__ __forceinline__ float mask_at(const ShapeArgs& sh, int x, int y, int z) {
  if (sh.kind == UR_SHAPE_ALL) return 1.f;
  const float dx = __fsub_rn((float)x, sh.cx);
  const float dy = __fsub_rn((float)y, sh.cy);
  const float dz = __fsub_rn((float)z, sh.cz);
  if (sh.kind == UR_SHAPE_SPHERE) {
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return d2 <= __fmul_rn(sh.s, sh.s) ? 1.f : 0.f;
  }
  float p[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    p[a] = fabsf(__fadd_rn(__fadd_rn(__fmul_rn(sh.r[a], dx), __fmul_rn(sh.r[3 + a], dy)), __fmul_rn(sh.r[6 + a], dz)));
  if (sh.kind == UR_SHAPE_CUBE) return (p[0] <= sh.s && p[1] <= sh.s && p[2] <= sh.s) ? 1.f : 0.f;
  return __fadd_rn(__fadd_rn(p[0], p[1]), p[2]) <= sh.s ? 1.f : 0.f;  // octahedron
}

// Per-row part of the predicate: the y and z terms are fixed along a row, so
// they are formed once (with the same roundings) and only the x term varies.
struct RowMask {
  int kind;
  float s, s2, dyz2;   // sphere: fl(dy*dy) and fl(dz*dz) folded below
  float dy2, dz2;
  float cx;
  float ry[3], rz[3];  // fl(R[1][a] dy), fl(R[2][a] dz)
  float r0[3];
  __device__ __forceinline__ void init(const ShapeArgs& sh, int y, int z) {
    kind = sh.kind;
    s = sh.s;
    s2 = __fmul_rn(sh.s, sh.s);
    cx = sh.cx;
    const float dy = __fsub_rn((float)y, sh.cy);
    const float dz = __fsub_rn((float)z, sh.cz);
    dy2 = __fmul_rn(dy, dy);
    dz2 = __fmul_rn(dz, dz);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      r0[a] = sh.r[a];
      ry[a] = __fmul_rn(sh.r[3 + a], dy);
      rz[a] = __fmul_rn(sh.r[6 + a], dz);
    }
  }
  // True when the mask is zero at every x of the row.  Sphere only: rounding
  // to nearest is monotone and fl(dx*dx) >= 0, so fl(fl(fl(dx*dx) + dy2) + dz2)
  // >= fl(dy2 + dz2) for every x; other shapes report false (no shortcut).
  __device__ __forceinline__ bool empty() const {
    return kind == UR_SHAPE_SPHERE && __fadd_rn(dy2, dz2) > s2;
  }
  __device__ __forceinline__ float at(int x) const {
    if (kind == UR_SHAPE_ALL) return 1.f;
    const float dx = __fsub_rn((float)x, cx);
    if (kind == UR_SHAPE_SPHERE) return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), dy2), dz2) <= s2 ? 1.f : 0.f;
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = fabsf(__fadd_rn(__fadd_rn(__fmul_rn(r0[a], dx), ry[a]), rz[a]));
    if (kind == UR_SHAPE_CUBE) return (p[0] <= s && p[1] <= s && p[2] <= s) ? 1.f : 0.f;
    return __fadd_rn(__fadd_rn(p[0], p[1]), p[2]) <= s ? 1.f : 0.f;
  }
};

// Sphere row (y, z) outside the particle: the test of RowMask::empty with the same
// roundings, for kernels that hold no RowMask.
__device__ __forceinline__ bool sphere_row_empty(const ShapeArgs& sh, int y, int z) {
  const float dy = __fsub_rn((float)y, sh.cy), dz = __fsub_rn((float)z, sh.cz);
  return __fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dz, dz)) > __fmul_rn(sh.s, sh.s);
}

// Rotated lattice (Sec. 2.3: the cell sampled on rotated planes with periodic wrap).
// Sample point of voxel (x, y, z) in cell-voxel units: p = R (x - c) + q, c = the shape
// centre; value: trilinear interpolation of the periodic cell at p.  Every product, sum
// and difference is rounded separately in the order below, so the result is the same
// float32 value on every device and in the reference of the tests.
struct LatArgs {
  int on;
  float r[9];
  float q[3];
};

__device__ __forceinline__ int ur_wrap(int i, int U) {
  int m = i % U;
  return m < 0 ? m + U : m;
}

__device__ __forceinline__ float ur_lerp(float a, float b, float f) { return __fadd_rn(a, __fmul_rn(f, __fsub_rn(b, a))); }

__device__ __forceinline__ float lattice_sample(const LatArgs& L, const ShapeArgs& sh, const float* __restrict__ cell,
                                                int U, int x, int y, int z) {
  const float d0 = __fsub_rn((float)x, sh.cx), d1 = __fsub_rn((float)y, sh.cy), d2 = __fsub_rn((float)z, sh.cz);
  float p[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    p[a] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(L.r[3 * a], d0), __fmul_rn(L.r[3 * a + 1], d1)),
                               __fmul_rn(L.r[3 * a + 2], d2)),
                     L.q[a]);
  int i0[3], i1[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float fl = floorf(p[a]);
    f[a] = __fsub_rn(p[a], fl);
    i0[a] = ur_wrap((int)fl, U);
    i1[a] = i0[a] + 1 == U ? 0 : i0[a] + 1;
  }
  // cell[z][y][x]; axis 0 = x
  const float* c00 = cell + ((long long)i0[2] * U + i0[1]) * U;
  const float* c01 = cell + ((long long)i0[2] * U + i1[1]) * U;
  const float* c10 = cell + ((long long)i1[2] * U + i0[1]) * U;
  const float* c11 = cell + ((long long)i1[2] * U + i1[1]) * U;
  const float v00 = ur_lerp(__ldg(c00 + i0[0]), __ldg(c00 + i1[0]), f[0]);
  const float v01 = ur_lerp(__ldg(c01 + i0[0]), __ldg(c01 + i1[0]), f[0]);
  const float v10 = ur_lerp(__ldg(c10 + i0[0]), __ldg(c10 + i1[0]), f[0]);
  const float v11 = ur_lerp(__ldg(c11 + i0[0]), __ldg(c11 + i1[0]), f[0]);
  return ur_lerp(ur_lerp(v00, v01, f[1]), ur_lerp(v10, v11, f[1]), f[2]);
}

static inline LatArgs ur_lattice_args(const ur_lattice* lat) {
  LatArgs L;
  memset(&L, 0, sizeof L);
  if (!lat) return L;
  L.on = 1;
  for (int i = 0; i < 9; ++i) L.r[i] = lat->rot[i];
  for (int i = 0; i < 3; ++i) L.q[i] = lat->offset[i];
  return L;
}

static inline ShapeArgs ur_shape_args(const ur_shape* shape) {
  ShapeArgs sh;
  sh.kind = shape->kind;
  sh.cx = shape->center[0];
  sh.cy = shape->center[1];
  sh.cz = shape->center[2];
  sh.s = shape->size;
  for (int i = 0; i < 9; ++i) sh.r[i] = shape->rot[i];
  return sh;
}
