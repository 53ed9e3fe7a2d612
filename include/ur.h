/*
 * ur.h -- C ABI of the GB300 wide-range X-ray scattering hot path.
 *
 * The operations follow "Ultima Ratio: simulating wide-range X-ray scattering
 * and diffraction" (Pauw et al., arXiv 2303.13435):
 *   ur_build_density  Sec. 2.3: ED-1 = unit cell tiled with periodic wrap and
 *                     multiplied by the particle mask; ED-2/ED-3 = block
 *                     integration with zero padding ("zoom out").
 *   ur_fft_intensity  Sec. 2.4 Eq. 1/Eq. 2: 3D transform split into 2D plane
 *                     transforms (only planes holding density) and 1D column
 *                     transforms (absent planes are zeros); I = |F|^2;
 *                     Sec. 2.5: isotropic averaging of I into Q bins.
 *   ur_bin_q          Sec. 2.5 averaging of a stored half-spectrum intensity.
 *   ur_merge          Sec. 2.5 (last paragraph) and Fig. 2: the per-level curves
 *                     combined into one absolute-scale I(Q).
 *   ur_backward       Not in the paper: the adjoint of the forward map, from
 *                     dL/d(bin mean) to dL/d(unit cell) and dL/d(mask weight).
 *   ur_batch_*        Many particles of uneven grid sizes in one launch sequence.
 *
 * Conventions (all calls):
 *   - Grids are cubic, edge N (even, 8 <= N <= 4096, N/2 a product of 2,3,5,7).
 *     A density is plane-major rho[z][y][x], x contiguous ("planes" are fixed z).
 *   - Spectra use the half axis along x: F[kz][ky][kx], kx in [0, N/2],
 *     complex64 (float2) interleaved, kx contiguous.  Axis index i has the
 *     signed frequency i (i < N/2) or i - N.  F follows Eq. 1 (1/N^3).
 *   - |Q| = dq sqrt(k^2), dq = 2 pi / (N dx) (nm^-1), evaluated in IEEE float64;
 *     bins are half-open [e_j, e_j+1), the last bin closed.
 *   - Bin statistics are double[UR_BIN_FIELDS][B] (field-major):
 *       [0] count  voxels of the full N^3 grid in the bin (integer-valued)
 *       [1] sum of I       [2] sum of I^2      [3] sum of |Q|
 *       [4] mean I (NaN when count = 0)
 *       [5] standard error of the mean (NaN when count < 2)
 *   - Pointers are device pointers unless the argument says "host".  The
 *     caller owns every buffer; the library owns only ur_plan objects (twiddle
 *     and bin tables) and allocates nothing else.  Work is queued on `stream`
 *     (a cudaStream_t; NULL = legacy default stream) and returns before it is
 *     done unless stated.
 *   - Every call returns a ur_status; on failure ur_last_error() gives a
 *     message (per thread).  No call aborts the process.
 */
#ifndef UR_H
#define UR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  UR_OK = 0,
  UR_ERR_INVALID = 1,        /* bad argument: sizes, alignment, null pointer */
  UR_ERR_OOM = 2,            /* pinned/device allocation inside plan creation failed */
  UR_ERR_CUDA = 3,           /* a CUDA runtime call failed; message has the CUDA error */
  UR_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up */
  UR_ERR_UNSUPPORTED = 5,    /* valid request this build does not implement */
  UR_ERR_FAULT_INJECTED = 6  /* host-side fault injection (UR_FAULT env) fired */
} ur_status;

enum { UR_F32 = 0, UR_F16 = 1 };

enum {
  UR_SHAPE_SPHERE = 0,      /* (dx*dx + dy*dy) + dz*dz <= s*s */
  UR_SHAPE_CUBE = 1,        /* max_a |p_a| <= s, p = R^T d */
  UR_SHAPE_OCTAHEDRON = 2,  /* (|p_0| + |p_1|) + |p_2| <= s */
  UR_SHAPE_ALL = 3,         /* no mask */
  UR_SHAPE_WEIGHTS = 4      /* per-voxel float32 weights array */
};

enum { UR_BIN_FIELDS = 6 };
enum { UR_BIN_COUNT = 0, UR_BIN_SUM_I = 1, UR_BIN_SUM_I2 = 2, UR_BIN_SUM_Q = 3, UR_BIN_MEAN = 4, UR_BIN_SEM = 5 };

/* Last error message of the calling thread ("" if none).  Never NULL. */
const char* ur_last_error(void);
const char* ur_version(void);

/* ---------------------------------------------------------------------------
 * Plans.  A plan fixes the grid, the ED storage type, the slab of planes that
 * hold density, and the Q bins.  Creation is synchronous: it allocates and
 * fills the plan's device tables (twiddles exp(-2 pi i t/N) generated in
 * float64 and rounded to float32; integer k^2 thresholds of the bins; the
 * data-independent per-bin count and sum of |Q|) on the current device.
 * ------------------------------------------------------------------------- */
typedef struct ur_plan ur_plan;

typedef struct {
  int32_t n;         /* grid edge N */
  double dx;         /* voxel edge, nm (> 0) */
  int32_t ed_dtype;  /* UR_F32 or UR_F16: element type of the ED read by ur_fft_intensity */
  int32_t z0;        /* first plane that may hold density */
  int32_t nz;        /* number of planes [z0, z0+nz) that may hold density; all others are zero (Sec. 2.4: skipped slices) */
} ur_grid_desc;

/* edges: host float64[nbins+1], strictly increasing, nm^-1; copied. */
ur_status ur_plan_create(const ur_grid_desc* grid, const double* edges, int32_t nbins, ur_plan** out);
ur_status ur_plan_destroy(ur_plan* plan);

/* Bin thresholds: host int64[nbins+1] out; bin j holds k^2 in [t_j, t_j+1). */
ur_status ur_plan_thresholds(const ur_plan* plan, int64_t* thresholds_out);

/* The same table without a plan (host only, no GPU needed), Sec. 2.5 bin
 * assignment: t_j = min{s >= 0 : dq sqrt(s) >= e_j} (j < B),
 * t_B = min{s : dq sqrt(s) > e_B}, dq = 2 pi/(N dx), in IEEE float64.
 * Values above 3 (N/2)^2 mean "beyond every voxel of the grid". */
ur_status ur_bin_thresholds(int32_t n, double dx, const double* edges, int32_t nbins, int64_t* thresholds_out);

/* Host-side failure injection (tests): UR_FAULT="<site>:<k>" in the
 * environment makes the k-th pass through <site> (plan_create,
 * fft_intensity, backward, host_slab) fail with UR_ERR_FAULT_INJECTED;
 * ur_fault_reset() re-reads the variable.  Nothing on the device is faulted. */
void ur_fault_reset(void);

enum { UR_WS_FORWARD = 1, UR_WS_BACKWARD = 2, UR_WS_HOST_SLABS = 4, UR_WS_ADJ_SLABS = 8 };
/* Workspace bytes for the operations in `what` (bitwise OR of UR_WS_*).
 * The forward workspace holds the plane-transform intermediate
 * (nz * N * (N/2+1) complex64) and the per-block bin partials; the backward
 * adds the inverse intermediate (N * N * (N/2+1) complex64).  UR_WS_HOST_SLABS
 * adds two staging slabs for ED read from pinned host memory.  UR_WS_ADJ_SLABS
 * (ur_backward_slabs) adds, after the forward part and the host staging slabs
 * (counted whether or not UR_WS_HOST_SLABS is given), one slab of the inverse
 * intermediate (ur_plan_set_adj_slab_planes planes) and two dL/dm staging
 * buffers of min(64, that) planes. */
size_t ur_workspace_size(const ur_plan* plan, int32_t what);

/* Planes per host->device slab of the out-of-core path (default: about
 * 256 MiB of ED per slab).  Changes ur_workspace_size(plan, UR_WS_HOST_SLABS). */
ur_status ur_plan_set_slab_planes(ur_plan* plan, int32_t planes);

/* Planes per chunk of the power-of-two path.  With chunks, the row pass and the
 * y-column pass of one chunk of planes run back to back so that the chunk's
 * intermediate is re-read from L2, and the adjoint's y-inverse of a chunk goes
 * to a chunk buffer that its row pass reads from L2.  Default: N (every pass is
 * one launch over all planes and the adjoint's y-inverse runs in place; no
 * chunk buffer).  planes >= 1 (clamped to N).  Changes ur_workspace_size(plan,
 * UR_WS_BACKWARD); results do not depend on it beyond rounding order.
 * ur_plan_chunk_planes returns the current value (0 for the runtime-radix path,
 * which does not chunk). */
ur_status ur_plan_set_chunk_planes(ur_plan* plan, int32_t planes);
int32_t ur_plan_chunk_planes(const ur_plan* plan);

/* Voxel-sinc correction of the binned intensity (Sec. 2.5 last paragraph: the
 * pattern taken with the voxel-sized sinc for better high-Q behaviour, left out
 * by the paper for its tiny voxels).  Reading: the voxelised density is a sum
 * of uniform cubes of edge dx, whose form factor multiplies the transform, so
 * with the option on every binned intensity is |F_k|^2 times
 * S(k) = prod_a sinc^2(pi k_a / N) (sinc x = sin x / x).  It brings the zoom
 * levels of ur_merge into agreement below each coarse level's limit (for a
 * density that is constant on the coarse voxels, exactly).  The plan keeps a
 * table of sinc^2(pi m / N) (float64-built, stored float32).  Counts and sum |Q|
 * are unchanged.  The adjoint (ur_backward, batches with an adjoint) rejects
 * such plans with UR_ERR_UNSUPPORTED.  ur_plan_voxel_sinc returns 1 when on. */
ur_status ur_plan_set_voxel_sinc(ur_plan* plan, int32_t on);
int32_t ur_plan_voxel_sinc(const ur_plan* plan);

/* Engine of the binned z pass for N = 256 and 512 (at most 1024 bins): 0 (the
 * default) = the compile-time register/shared-memory kernel; 1 = a persistent
 * kernel that stages 16-column tiles with TMA (cp.async.bulk.tensor, mbarrier
 * completion, waits bounded to about a second) and transforms each column with
 * one warp-local exchange.  Both give the same statistics (per-bin shifted sums
 * merged in FP64); the TMA engine measured slower at 512^3 (its 128 registers
 * and 111 KB of shared memory per block leave 16 warps per SM).  Other plans get
 * UR_ERR_UNSUPPORTED for 1.  ur_plan_tma_zpass returns the setting. */
ur_status ur_plan_set_tma_zpass(ur_plan* plan, int32_t on);
int32_t ur_plan_tma_zpass(const ur_plan* plan);

/* ---------------------------------------------------------------------------
 * ur_build_density (Sec. 2.3).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t kind;       /* UR_SHAPE_* */
  float center[3];    /* (x, y, z) particle centre in voxel-index units */
  float size;         /* sphere radius, cube half-edge, octahedron vertex distance; voxels */
  float rot[9];       /* row-major R; body coordinates p = R^T d, d = (x, y, z) - centre */
} ur_shape;

/* ED-1: rho[z][y][x] = fl32(u[(z+oz)%U][(y+oy)%U][(x+ox)%U] * m(x,y,z)) for
 * planes z in [z_begin, z_begin+z_count), written plane-major to ed_out
 * (z_count*N*N elements of out_dtype, FP16 rounded to nearest even).
 *   cell     device float32[U][U][U]
 *   origin   host int32[3] (ox, oy, oz), tiling offset, >= 0
 *   shape    host; kind UR_SHAPE_WEIGHTS reads weights (device float32 N^3,
 *            full box, plane-major) instead of a predicate.
 *   nz_range device int32[2] or NULL: atomically lowered/raised to the
 *            first/last plane written with a nonzero voxel; the caller
 *            initialises it to {INT32_MAX, -1}.
 * The mask decision is taken in float32 with separately rounded products and
 * sums in the order written above (no fused multiply-add). */
ur_status ur_build_density(int32_t n, const float* cell, int32_t ucell, const int32_t* origin,
                           const ur_shape* shape, const float* weights, int32_t z_begin,
                           int32_t z_count, int32_t out_dtype, void* ed_out, int32_t* nz_range,
                           void* stream);

/* Rotated lattice (Sec. 2.3 first paragraph: the cell interpolated over rotated
 * planes with the cell repeated outside its bounds, the route to crystallites
 * of any orientation).  Voxel (x, y, z) samples the cell at the cell-voxel
 * coordinate p = R (x - c) + q, c = the shape's centre, by trilinear
 * interpolation of the periodic cell (order 1).  Every product, sum and
 * difference is rounded separately in float32, in the order
 * p_a = ((R[a][0] d_0 + R[a][1] d_1) + R[a][2] d_2) + q_a with d = (x, y, z) - c;
 * i = floor(p), f = p - i; lerp(a, b, f) = a + f (b - a) along x, then y, then z
 * over the neighbours (i + {0, 1}) mod U.  With R = I and an integer q the
 * samples are cell voxels: the integer wrap of ur_build_density with origin
 * q - c. */
typedef struct {
  float rot[9];     /* row-major R */
  float offset[3];  /* q, cell-voxel units */
} ur_lattice;

/* ur_build_density with the cell sampled on a rotated lattice (lattice
 * non-NULL; all other arguments as for ur_build_density, without an origin).
 * The adjoint (ur_backward) does not take a lattice. */
ur_status ur_build_density_lattice(int32_t n, const float* cell, int32_t ucell, const ur_lattice* lattice,
                                   const ur_shape* shape, const float* weights, int32_t z_begin, int32_t z_count,
                                   int32_t out_dtype, void* ed_out, int32_t* nz_range, void* stream);

/* ED-2/ED-3 (Sec. 2.3): out[Z][Y][X] = sum of src over the f^3 block at
 * (f Z', f Y', f X') where (Z', Y', X') = (Z, Y, X) - o, o = (n_out - n_src/f)/2,
 * and 0 outside the placed block; out is the full n_out^3 box.  FP16 sources
 * are summed exactly (integer multiples of 2^-24) and rounded once to the
 * output type; FP32 sources are summed in float64. */
ur_status ur_zoom_density(int32_t n_src, int32_t src_dtype, const void* src, int32_t f, int32_t n_out,
                          int32_t out_dtype, void* out, void* stream);

/* ---------------------------------------------------------------------------
 * ur_fft_intensity (Sec. 2.4-2.5).
 *   ed       the nz planes [z0, z0+nz) of the density, plane-major, ed_dtype.
 *            ed_on_host = 0: device pointer.  ed_on_host = 1: pinned host
 *            memory; planes are streamed to the device in slabs on an
 *            internal copy stream, double-buffered, overlapping the plane
 *            transforms (the workspace must include UR_WS_HOST_SLABS).
 *   bins     device double[UR_BIN_FIELDS][B] or NULL (no binning).
 *   F_out    device complex64 [N][N][N/2+1] (Eq. 1 normalised) or NULL.
 *   ws       device workspace of ur_workspace_size(plan, UR_WS_FORWARD [| UR_WS_HOST_SLABS]).
 *            The intermediate it holds is what ur_backward recomputes F from.
 * ------------------------------------------------------------------------- */
ur_status ur_fft_intensity(const ur_plan* plan, const void* ed, int32_t ed_on_host, double* bins,
                           void* F_out, void* ws, size_t ws_bytes, void* stream);

/* ur_fft_intensity with the density generated inside the plane pass
 * (Sec. 2.3 tile + mask fused with Sec. 2.4): the ED of planes
 * [z0, z0+nz) is never stored.  cell, ucell, origin, shape and weights are
 * as for ur_build_density; the transform sees exactly the values
 * ur_build_density would write (FP32).  The plan's ed_dtype is ignored.
 * Cell values must be finite: a row whose mask is zero everywhere (a sphere
 * row outside the particle, or any row whose generated values are all zero)
 * is taken as zero without evaluating u * 0. */
ur_status ur_fft_intensity_tiled(const ur_plan* plan, const float* cell, int32_t ucell, const int32_t* origin,
                                 const ur_shape* shape, const float* weights, double* bins, void* F_out, void* ws,
                                 size_t ws_bytes, void* stream);

/* ur_fft_intensity_tiled with the density of ur_build_density_lattice (the cell
 * sampled on a rotated lattice) generated inside the plane pass. */
ur_status ur_fft_intensity_tiled_lattice(const ur_plan* plan, const float* cell, int32_t ucell,
                                         const ur_lattice* lattice, const ur_shape* shape, const float* weights,
                                         double* bins, void* F_out, void* ws, size_t ws_bytes, void* stream);

/* ur_fft_intensity_noalloc -- the paper has no counterpart; this entry point
 * serves callers that must not allocate device memory while they run (a
 * real-time or embedded loop with a memory budget fixed at start-up, a
 * plugin whose host program owns all device allocations, or code that cannot
 * call the CUDA allocator).  It computes what ur_fft_intensity computes with
 * F_out = NULL, but keeps the plane-transform intermediate in a scratch
 * array built into the library instead of a caller workspace, and it calls no
 * allocator itself.  The plan is still created beforehand (that allocates
 * the plan's tables once).
 *   - Limit: the intermediate, nz * N * (N/2+1) * 8 bytes, must fit
 *     UR_NOALLOC_SCRATCH_BYTES (64 MiB); larger plans get UR_ERR_INVALID
 *     and a message naming both sizes.
 *   - Every GPU that loads the library reserves those 64 MiB until the
 *     process exits.
 *   - The first call on a device looks up the scratch array's device address
 *     (with that device current); make that first call before any stream
 *     capture.
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls whose work overlaps on the GPU (two streams at once) race and
 *     give wrong results; serialise them.
 *   - The current device must be the one the plan was created on
 *     (UR_ERR_INVALID otherwise).  The UR_FAULT site "fft_intensity" covers
 *     this call too.
 *   ed: device planes [z0, z0+nz), ed_dtype; bins: device double[6][B] (required). */
#define UR_NOALLOC_SCRATCH_BYTES (64u << 20)
ur_status ur_fft_intensity_noalloc(const ur_plan* plan, const void* ed, double* bins, void* stream);
/* Size of that scratch array in bytes, as built into the library (host only). */
size_t ur_noalloc_scratch_bytes(void);

/* Sec. 2.5 binning of a stored half-spectrum intensity I[kz][ky][kx]
 * (device float32, N*N*(N/2+1), Eq. 1 normalised); kx in (0, N/2) weighs 2
 * (the mirrored half), kx = 0 and N/2 weigh 1.  ws: ur_workspace_size(plan, UR_WS_FORWARD). */
ur_status ur_bin_q(const ur_plan* plan, const float* intensity_half, double* bins, void* ws,
                   size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ur_merge (Sec. 2.5 last paragraph; Fig. 2 caption; Sec. 2.7 for the
 * uncertainty-weighted combination of overlapping curves).
 *   nlev        number of levels (1..8)
 *   level_bins  host array of nlev device pointers, each double[UR_BIN_FIELDS][B]
 *               binned over the same edges
 *   level_n     host int32[nlev], grid edge of each level (intensity scale N^6)
 *   level_dx    host double[nlev], voxel edge of each level (nm); the library
 *               trusts a level up to Q_max/2 = pi/dx (ur_level_qmax), the
 *               artefact limit of the Fig. 2 caption with Q_max = 2 pi/dx
 *   edges       device double[B+1] (the edges all levels were binned on)
 *   mode        UR_MERGE_WINDOWS: disjoint windows.  Levels are ordered by
 *               their limit; the one with the smallest limit covers [0, its
 *               limit), each next one [previous limit, its limit), the last
 *               one closed.  Each output bin takes the level whose window
 *               holds sqrt(e_j e_j+1).
 *               UR_MERGE_INVVAR: each output bin combines every level trusted
 *               at sqrt(e_j e_j+1) that has voxels and a finite positive SEM
 *               there, with weights 1/SEM^2 (absolute units): mean = sum w m /
 *               sum w, SEM = (sum w)^(-1/2), count and sum |Q| added; bins with
 *               no such level fall back to the windows choice.
 *   out         device double[5][B]: mean, sem (absolute units, electrons^2),
 *               count, mean |Q|, source level (-1: none; INVVAR: the level of
 *               largest weight).
 * Errors: UR_ERR_INVALID for nlev outside [1, 8], null pointers, N <= 0, a dx
 * that is not finite and positive, or an unknown mode.
 * ------------------------------------------------------------------------- */
enum { UR_MERGE_WINDOWS = 0, UR_MERGE_INVVAR = 1 };
ur_status ur_merge(int32_t nlev, const double* const* level_bins, const int32_t* level_n,
                   const double* level_dx, const double* edges, int32_t nbins, int32_t mode, double* out,
                   void* stream);
/* The upper |Q| (nm^-1) up to which ur_merge trusts a level of voxel edge dx: pi/dx
 * (host only; 0 for a dx that is not finite and positive). */
double ur_level_qmax(double dx);

/* ---------------------------------------------------------------------------
 * Ewald-sphere detector image (Sec. 2.5 first paragraph: for anisotropic
 * samples, the 2D data of a practical experiment are the intensity read on the
 * Ewald sphere, a shell whose thickness the wavelength distribution sets).
 *   F_half  device complex64 [N][N][N/2+1], the F_out of ur_fft_intensity
 *           (Eq. 1 normalised)
 *   det     host; a flat detector normal to the beam (+z) at distance_m;
 *           pixel (ix, iy) at ((ix - beam_x) pixel_m, (iy - beam_y) pixel_m);
 *           nlambda wavelengths lambda_l = wavelength_nm (1 + bandwidth ((l +
 *           1/2)/nlambda - 1/2)) (uniform band of relative full width
 *           `bandwidth`, 1 <= nlambda <= 16); rot = sample orientation R
 *           (row-major), q_sample = R^T q_lab.
 *   image   device float32 [ny][nx]: per pixel the mean over wavelengths of
 *           |F|^2 at q = (2 pi / lambda)(s - z_hat) (s the unit vector to the
 *           pixel), trilinearly interpolated between the 8 neighbouring grid
 *           frequencies (F(-k) = conj F(k) for the missing half); samples whose
 *           neighbours leave [-N/2, N/2 - 1] are dropped; NaN where none is left.
 *           Eq. 1 units (times N^6 for electrons^2).  Geometry in float32.
 * Errors: UR_ERR_INVALID for null pointers, sizes outside range or a
 * non-positive pixel, distance or wavelength.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t nx, ny;
  double pixel_m, distance_m;
  double beam_x, beam_y;
  double wavelength_nm, bandwidth;
  int32_t nlambda;
  float rot[9];
} ur_detector;
ur_status ur_ewald_image(const ur_plan* plan, const void* F_half, const ur_detector* det, float* image, void* stream);

/* ---------------------------------------------------------------------------
 * Polydisperse ensemble (Sec. 3: broad polydispersity described by about 200
 * volume-weighted single-particle simulations, summed into one curve).
 *   count        number of particles (1..512)
 *   item_bins    host array of device pointers, each double[UR_BIN_FIELDS][B]
 *                over the same edges (e.g. the bins of a ur_batch)
 *   item_n       host int32[count], grid edge of each particle (scale N^6)
 *   weights      host double[count], w_i; volume weighting is w_i = phi_i / V_i
 *                (phi_i the volume fraction of the size class, V_i the volume)
 *   out          device double[4][B]: mean = sum_i w_i N_i^6 mean_ij (absolute
 *                units), SEM = sqrt(sum_i (w_i N_i^6 SEM_ij)^2), count, mean |Q|.
 *                A bin is NaN (count 0) unless every particle of nonzero
 *                weight has voxels in it.
 * ur_ensemble_backward scatters dL/d(ensemble mean) to each particle:
 * item_dl_dmean[i][j] = w_i N_i^6 dl_dens[j] on valid bins, 0 elsewhere (host
 * array of device pointers, each double[B], ready for ur_backward or a batch).
 * One kernel launch each; the tables are kernel parameters (capturable).
 * Errors: UR_ERR_INVALID for a count outside [1, 512], null pointers, N <= 0
 * or a weight that is not finite.
 * ------------------------------------------------------------------------- */
ur_status ur_ensemble(int32_t count, const double* const* item_bins, const int32_t* item_n, const double* weights,
                      int32_t nbins, double* out, void* stream);
ur_status ur_ensemble_backward(int32_t count, const double* const* item_bins, const int32_t* item_n,
                               const double* weights, int32_t nbins, const double* dl_dens,
                               double* const* item_dl_dmean, void* stream);

/* ---------------------------------------------------------------------------
 * ur_backward: adjoint of ur_build_density + ur_fft_intensity for a loss L
 * on the bin means (not in the paper).
 *   dl_dmean  device double[B], dL/d(mean I_j)
 *   fwd_bins  device double[UR_BIN_FIELDS][B] from the forward (counts)
 *   F         device complex64 half spectrum from the forward's F_out, or
 *             NULL: F is recomputed column by column from the forward
 *             intermediate still held in ws.
 *   cell, ucell, origin, shape, weights: as given to ur_build_density.
 *   dl_dcell  device float32[U][U][U] (overwritten)
 *   dl_dmask  device float32[N][N][N] (overwritten), or NULL
 *   ws        the forward's workspace, sized with UR_WS_FORWARD | UR_WS_BACKWARD.
 * dL/drho(x) = (2/N^3) Re sum_k G_k F_k exp(+2 pi i k.x/N), G_k = dl_dmean_j / count_j
 * on the voxels of bin j; dL/dm = dL/drho * u(x mod U); dL/du(c) = sum over the
 * tiles of dL/drho * m.
 * ------------------------------------------------------------------------- */
ur_status ur_backward(const ur_plan* plan, const double* dl_dmean, const double* fwd_bins, const void* F,
                      const float* cell, int32_t ucell, const int32_t* origin, const ur_shape* shape,
                      const float* weights, float* dl_dcell, float* dl_dmask, void* ws, size_t ws_bytes,
                      void* stream);

/* Out-of-core adjoint (the per-slab adjoint of config-sized grids whose inverse
 * intermediate of all N planes, N * N * (N/2+1) complex64, does not fit; the
 * paper's Sec. 2.4 slice-wise processing applied to the adjoint).  Same
 * result as ur_backward with F = NULL, computed slab by slab: for each slab of
 * adj_slab_planes output planes the z pass is recomputed over every spectrum
 * column from the forward intermediate in ws (recomputation instead of storing
 * F), and only the slab's planes go through the y inverse and the row pass.
 * dL/du accumulates on the device; dL/dm (optional) is written to
 * dl_dmask_host, pinned host float32 [N][N][N], in sub-slabs of up to 64 planes
 * by a copy stream overlapping the next rows (two device staging buffers).
 * Each slab rereads the whole forward intermediate, so fewer, larger slabs
 * cost less.  ws: the forward's workspace, sized
 * with UR_WS_FORWARD | UR_WS_ADJ_SLABS, still holding the forward intermediate.
 * Power-of-two grids only (UR_ERR_INVALID otherwise); plans with the voxel-sinc
 * correction get UR_ERR_UNSUPPORTED.  The caller's stream waits for the copies. */
ur_status ur_backward_slabs(const ur_plan* plan, const double* dl_dmean, const double* fwd_bins, const float* cell,
                            int32_t ucell, const int32_t* origin, const ur_shape* shape, const float* weights,
                            float* dl_dcell, float* dl_dmask_host, void* ws, size_t ws_bytes, void* stream);
/* Output planes per slab of ur_backward_slabs (default: about 4 GiB of inverse
 * intermediate); changes ur_workspace_size(plan, UR_WS_ADJ_SLABS). */
ur_status ur_plan_set_adj_slab_planes(ur_plan* plan, int32_t planes);

/* Log-I(Q) mean-squared error against a target curve and its gradient, the
 * loss of the batched workload and of the benchmark step (not in the paper;
 * the fit of a simulated curve to a measured one that Sec. 3 motivates):
 *   L = (1/V) sum over valid bins of (ln mean_j - ln target_j)^2, valid = finite
 *   and positive mean, V = max(number of valid bins, 1);
 *   dl_dmean_j = 2 (ln mean_j - ln target_j) / (mean_j V) on valid bins, else 0.
 * bins: device double[UR_BIN_FIELDS][nbins] from a forward; target: device
 * double[nbins] (positive where bins are valid); loss: device double[1] or NULL;
 * dl_dmean: device double[nbins] (overwritten), ready for ur_backward.  One
 * kernel launch (plus a memset of *loss), float64 throughout; L is summed over
 * blocks with atomics, so its last bits may depend on scheduling; nbins <= 8192
 * (UR_ERR_INVALID above). */
ur_status ur_log_mse_grad(int32_t nbins, const double* bins, const double* target, double* loss, double* dl_dmean,
                          void* stream);

/* Completion status of the work queued so far on `stream`: waits for it
 * (host blocks) and returns UR_OK, or UR_ERR_CUDA with the CUDA error in
 * ur_last_error() when a kernel or copy on the device failed.  The library's
 * kernels contain no device-side waits, so there are no timeout words to
 * report; UR_ERR_TIMEOUT stays reserved for such waits. */
ur_status ur_sync_status(void* stream);

/* Per-thread event timing of the last ur_fft_intensity on this thread
 * (milliseconds per internal kernel, in launch order); for measurement only.
 * Enabled by ur_set_timing(1).  Returns the number of entries written. */
void ur_set_timing(int32_t enable);
int32_t ur_last_timings(float* ms_out, int32_t max_entries, const char** names_out);

/* ---------------------------------------------------------------------------
 * Batched particles of uneven grid sizes (Sec. 3: polydispersity as many
 * particle simulations).  A batch is built once from its items; afterwards
 * ur_batch_forward runs the tiled forward (density generated in the plane
 * pass, transform, |F|^2, bins) of every item and ur_batch_backward the adjoint
 * of every item, each as a fixed sequence of five kernel launches whose
 * blocks cover all items (no host work in between, so the pair can be
 * captured in one CUDA graph).  Items keep their buffers for the life of the
 * batch.  The batch uses the runtime-radix kernels for every grid edge.
 * ------------------------------------------------------------------------- */
typedef struct ur_batch ur_batch;
typedef struct {
  const ur_plan* plan;     /* grid, plane slab and bins of this particle */
  const float* cell;       /* device float32 U^3 */
  int32_t ucell;
  int32_t origin[3];
  ur_shape shape;
  const float* weights;    /* device N^3, UR_SHAPE_WEIGHTS only */
  double* bins;            /* device double[UR_BIN_FIELDS][B]: forward output */
  void* ws;                /* device workspace, 256-byte aligned */
  size_t ws_bytes;         /* >= ur_workspace_size(plan, UR_WS_FORWARD | UR_WS_BACKWARD) (FORWARD only without adjoint) */
  const double* dl_dmean;  /* device double[B]: adjoint input, or NULL (no adjoint) */
  float* dl_dcell;         /* device float32 U^3: adjoint output, or NULL */
  float* dl_dmask;         /* device float32 N^3: adjoint output, or NULL */
} ur_batch_item;

ur_status ur_batch_create(int32_t count, const ur_batch_item* items, ur_batch** out);
ur_status ur_batch_destroy(ur_batch* batch);
ur_status ur_batch_forward(const ur_batch* batch, void* stream);
ur_status ur_batch_backward(const ur_batch* batch, void* stream);

/* Tile shape of the runtime-radix kernels of a plan (the autotuner's knob):
 * rows per block of the row passes and columns per block of the column
 * passes; 0 keeps the current value.  rows * N/2 and cols * N must not exceed
 * 4096 (elements held by a 256-thread block).  Takes effect for later calls
 * and for batches created afterwards. */
ur_status ur_plan_set_tiles(ur_plan* plan, int32_t rows_per_block, int32_t cols_per_block);
ur_status ur_plan_get_tiles(const ur_plan* plan, int32_t* rows_per_block, int32_t* cols_per_block);

#ifdef __cplusplus
}
#endif
#endif /* UR_H */
