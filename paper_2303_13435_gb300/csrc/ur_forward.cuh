// Declarations shared by the forward, adjoint, out-of-core and batched
// translation units.
#pragma once

#include "ur_common.cuh"
#include "ur_density.cuh"

#define UR_EMAX 16  // elements per thread in the shared-memory FFT engine

enum { COL_Y = 0, COL_ZBIN = 1, COL_ZADJ = 2 };

__host__ __device__ inline size_t ur_align_up_dev(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct ColArgs {
  const float2* src;
  float2* dst;
  long long ncols;
  int N, H, M;
  long long A;       // source offset per outer index (c / H)
  long long S;       // source stride between column elements
  long long Ad, Sd;  // destination offset per outer index / element stride
  int nload;         // elements per column read from src
  int zoff;          // position of the first loaded element in the column
  int TX;            // columns per block
  int pitch;         // shared-memory pitch between columns (float2)
  const StageInfo* sched;
  int nst;
  const float2* tw;
  const float2* stw;   // stage twiddles of the N-point transform (power-of-two kernels)
  // binning
  const int32_t* thr;
  const int16_t* lut;  // k^2 -> bin (-1 outside)
  const int16_t* crs;  // coarse rank table of k^2 (UR_COARSE_ENTRIES, bin_rank)
  int crs_shift;
  int nbins;
  float iscale;      // I' = |F~|^2 * iscale (I' = N^3 I)
  const float* vs;   // voxel-sinc factors sinc^2(pi m / N), m = 0..N/2, or NULL (binning of plain |F|^2)
  double* gsum;      // [nbins] sum of w I' (shifted kernels: of w (I' - K_j))
  double* gsum2;     // [nbins] sum of w I'^2 (shifted kernels: of w (I' - K_j)^2)
  unsigned long long* gK;  // shifted kernels: per-bin shift K_j, set once by the first block that
                           // reaches the bin (0 = unset; else (1 << 32) | float bits)
  float2* fout;      // optional F half spectrum [kz][ky][kx]
  float fscale;
  // adjoint
  const float* sigma;  // per-bin scale of F~ along z (adjoint)
  int skip_fwd;        // 1: the loaded column is already the spectrum along z
  int row_skip;        // power-of-two forward y pass over a generated sphere density: rows
  int gen_z0;          // (y, gen_z0 + plane) outside the sphere are zero and were not
  ShapeArgs sh;        // written by the row pass; they are not read
  int out_lo, out_cnt; // adjoint z pass: write only the planes z in [out_lo, out_lo + out_cnt), at
                       // z - out_lo (out_cnt = 0: every plane)
  int k2_zero;         // power-of-two adjoint: spectrum columns with kx^2 + ky^2 >= k2_zero are
                       // zero; the z pass may leave them unwritten and the y pass does not read
                       // them (0x7fffffff: none)
};

// generic adjoint row pass (one block: a batch of rows wrapping onto one cell row)
struct GenGradArgs {
  const float2* Y;
  int N, RB, nst;
  const StageInfo* sched;
  const float2* tw;
  const float* cell;
  int U, ox, oy, oz;
  ShapeArgs sh;
  const float* weights;
  float inv_n3;
  float* dl_dmask;
  float* dl_dcell;
};

// ---------------------------------------------------------------------------
// Batched launches: one grid covers the blocks of every item; block b belongs
// to item i with start[i] <= b < start[i+1] (device tables built once).
// ---------------------------------------------------------------------------
struct RowArgs;
struct BatchRowsItem;
struct BatchFinItem {
  double* bins;
  const double* geo;
  int nb;
  double inv_n3;
};
struct BatchSigmaItem {
  const double* g;
  const double* bins;
  int nb;
  double n3;
  float* sigma;
};
struct BatchZeroItem {
  void* ptr;
  size_t bytes;
};
struct BatchGradItem {
  GenGradArgs g;
  int gx;  // blocks along the row batches of one cell row
};

ur_status ur_batch_launch_rows(const BatchRowsItem* items, const long long* start, int count, long long nblocks,
                               size_t smem, cudaStream_t s);
ur_status ur_batch_launch_cols(int mode, bool inv, const ColArgs* items, const long long* start, int count,
                               long long nblocks, size_t smem, cudaStream_t s);
ur_status ur_batch_launch_finalize(const BatchFinItem* items, int count, int maxnb, cudaStream_t s);
ur_status ur_batch_launch_sigma(const BatchSigmaItem* items, int count, int maxnb, cudaStream_t s);
ur_status ur_batch_launch_zero(const BatchZeroItem* items, int count, cudaStream_t s);
ur_status ur_batch_launch_grad(const BatchGradItem* items, const long long* start, int count, long long nblocks,
                               size_t smem, cudaStream_t s);

ColArgs ur_col_args(const ur_plan* p);
ur_status ur_plane_pass(const ur_plan* p, const void* ed, long long nplanes, float2* X, cudaStream_t s);
ur_status ur_column_pass(const ur_plan* p, const float2* X, double* bins, float2* F_out, cudaStream_t s);
ur_status ur_fft_intensity_host(const ur_plan* p, const void* ed_host, double* bins, float2* F_out, void* ws,
                                size_t ws_bytes, cudaStream_t s);
ur_status ur_launch_cols(int mode, bool inv, const ur_plan* p, const ColArgs& a, int grid, size_t smem, cudaStream_t s);

// per-kernel event timing (enabled by ur_set_timing)
void ur_timing_begin(const char* name, cudaStream_t s);
void ur_timing_end(cudaStream_t s);
