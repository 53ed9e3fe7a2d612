// Argument blocks and host entry points of the power-of-two kernels.
#pragma once

#include "ur_forward.cuh"
#include "ur_density.cuh"

// Values per thread of the power-of-two column transforms of length n: 16 from 1024 on
// (three radix-16 stages at 4096 instead of four radix-8 ones; measured 22-23 % faster
// steps at 1024-4096), 8 below (16 was 17 % slower at 512: half the resident warps).
#define UR_FAST_COL_E(n) ((n) >= 1024 ? 16 : 8)

struct RowArgs {
  const void* ed;          // density rows (GEN = 0), plane-major, nrows x N
  float2* X;               // output half-spectrum rows, nrows x (N/2+1)
  long long nrows;
  int z0;                  // absolute plane index of row 0 / N (GEN = 1)
  const float* cell;       // GEN = 1: unit cell U^3
  int ucell, ox, oy, oz;   // origin >= 0
  FastDiv fu;              // division by ucell
  ShapeArgs sh;
  LatArgs lat;             // GEN = 2: the cell sampled on a rotated lattice
  const float* weights;    // GEN >= 1 with UR_SHAPE_WEIGHTS: full-box weights
  const float2* tw;        // table exp(-2 pi i t / N), t < N
  const float2* stw;       // stage twiddles of the N/2-point transform (power-of-two kernels)
  int skip_empty;          // GEN = 1, sphere, N <= 512: rows outside the particle are not written
};

struct GradArgs {
  const float2* Y;         // inverse-transformed rows (along z and y), planes [ybase_z, ...)
  int ybase_z;
  int z0;                  // first absolute plane of this launch
  int rb;                  // rows per block (set by the launcher)
  const float2* tw;
  const float2* stw;       // stage twiddles of the N/2-point transform
  const float* cell;
  int ucell, ox, oy, oz;   // origin, each reduced to [0, ucell) by the host
  int cstep;               // (N/8) mod ucell (set by the launcher)
  ShapeArgs sh;
  const float* weights;
  float inv_n3;
  float* dl_dmask;         // dL/dm planes from mbase_z on (plane z at z - mbase_z)
  int mbase_z;
  float* dl_dcell;
};

// one item of a batched generic row pass
struct BatchRowsItem {
  RowArgs ra;
  int N, RB, nst, gen;
  const StageInfo* sched;
};

bool ur_fast_supported(int n);
ur_status ur_fast_rows(int n, const RowArgs& a, int gen, int ed_f16, cudaStream_t s);
ur_status ur_fast_cols(int n, int mode, const ColArgs& a, cudaStream_t s);
ur_status ur_fast_rows_grad(int n, const GradArgs& a, int nplanes, cudaStream_t s);
