// Host side of libur: errors, fault injection, plans (twiddles, bin tables,
// launch configuration), workspace sizes, and the level merge.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>

#include "ur_fast.cuh"

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[1024] = "";

void ur_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

extern "C" const char* ur_last_error(void) { return g_err; }
extern "C" const char* ur_version(void) { return "libur 0.1 (sm_103a)"; }

// Host-side fault injection for failure-path tests: UR_FAULT="<site>:<k>"
// makes the k-th (1-based) pass through fault point <site> fail with
// UR_ERR_FAULT_INJECTED.  Nothing on the device is faulted.
static std::mutex g_fault_mu;
static std::string g_fault_site;
static long g_fault_target = -1;
static long g_fault_count = 0;
static bool g_fault_loaded = false;

ur_status ur_fault_point(const char* site) {
  std::lock_guard<std::mutex> lk(g_fault_mu);
  if (!g_fault_loaded) {
    g_fault_loaded = true;
    const char* env = getenv("UR_FAULT");
    if (env && *env) {
      const char* colon = strrchr(env, ':');
      if (colon) {
        g_fault_site.assign(env, colon - env);
        g_fault_target = atol(colon + 1);
      } else {
        g_fault_site = env;
        g_fault_target = 1;
      }
    }
  }
  if (g_fault_target > 0 && g_fault_site == site) {
    if (++g_fault_count == g_fault_target) {
      ur_set_error("fault injected at %s (pass %ld)", site, g_fault_count);
      return UR_ERR_FAULT_INJECTED;
    }
  }
  return UR_OK;
}

extern "C" ur_status ur_sync_status(void* stream) {
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    ur_set_error("ur_sync_status: %s", cudaGetErrorString(e));
    return UR_ERR_CUDA;
  }
  // bounded device-side waits that gave up leave a word behind
  return ur_deverr_take();
}

extern "C" void ur_fault_reset(void) {
  std::lock_guard<std::mutex> lk(g_fault_mu);
  g_fault_loaded = false;
  g_fault_site.clear();
  g_fault_target = -1;
  g_fault_count = 0;
}

// ---------------------------------------------------------------------------
// Per-kernel event timing (measurement aid; off by default).  Each internal
// launch is bracketed by two events on its own stream; ur_last_timings waits
// for them and reports the accumulated entries of the calling thread.
// ---------------------------------------------------------------------------
struct TimingSlot {
  const char* name;
  cudaEvent_t a, b;
};
static thread_local bool g_timing = false;
static thread_local TimingSlot* g_slots = nullptr;
static thread_local int g_nslots = 0, g_used = 0;

extern "C" void ur_set_timing(int32_t enable) {
  g_timing = enable != 0;
  g_used = 0;
}

void ur_timing_begin(const char* name, cudaStream_t s) {
  if (!g_timing) return;
  if (g_used == g_nslots) {
    int nn = g_nslots ? 2 * g_nslots : 64;
    TimingSlot* ns = (TimingSlot*)realloc(g_slots, sizeof(TimingSlot) * nn);
    if (!ns) return;
    for (int i = g_nslots; i < nn; ++i) {
      cudaEventCreate(&ns[i].a);
      cudaEventCreate(&ns[i].b);
    }
    g_slots = ns;
    g_nslots = nn;
  }
  g_slots[g_used].name = name;
  cudaEventRecord(g_slots[g_used].a, s);
}

void ur_timing_end(cudaStream_t s) {
  if (!g_timing || g_used >= g_nslots) return;
  cudaEventRecord(g_slots[g_used].b, s);
  ++g_used;
}

extern "C" int32_t ur_last_timings(float* ms_out, int32_t max_entries, const char** names_out) {
  int n = 0;
  for (int i = 0; i < g_used && n < max_entries; ++i, ++n) {
    cudaEventSynchronize(g_slots[i].b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g_slots[i].a, g_slots[i].b);
    if (ms_out) ms_out[n] = ms;
    if (names_out) names_out[n] = g_slots[i].name;
  }
  g_used = 0;
  return n;
}

// ---------------------------------------------------------------------------
// Radix schedules
// ---------------------------------------------------------------------------
bool ur_make_sched(int L, int n_tab, Sched* out) {
  memset(out, 0, sizeof *out);
  out->L = L;
  // prime exponents, then few stages from the kernels' radices: 8s, a leftover 2
  // merged with a 3 or a 5 (6, 10), pairs of 3s as 9.  Fewer stages mean fewer
  // shared-memory round trips.
  int e2 = 0, e3 = 0, e5 = 0, e7 = 0;
  int r = L;
  while (r % 2 == 0) { ++e2; r /= 2; }
  while (r % 3 == 0) { ++e3; r /= 3; }
  while (r % 5 == 0) { ++e5; r /= 5; }
  while (r % 7 == 0) { ++e7; r /= 7; }
  if (r != 1 || L < 1 || n_tab % L != 0) return false;
  int cnt[UR_NRADIX] = {0};  // per entry of ur_radix_order
  auto add = [&](int R) {
    for (int i = 0; i < UR_NRADIX; ++i)
      if (ur_radix_order[i] == R) ++cnt[i];
  };
  for (; e2 >= 3; e2 -= 3) add(8);
  if (e2 == 2) {
    add(4);
  } else if (e2 == 1) {
    if (e3 > 0) { add(6); --e3; }
    else if (e5 > 0) { add(10); --e5; }
    else add(2);
  }
  for (; e3 >= 2; e3 -= 2) add(9);
  if (e3 == 1) add(3);
  for (; e5 > 0; --e5) add(5);
  for (; e7 > 0; --e7) add(7);
  int rad[64];
  int nr = 0;
  for (int i = 0; i < UR_NRADIX; ++i)
    for (int c = 0; c < cnt[i]; ++c) rad[nr++] = ur_radix_order[i];
  if (nr > UR_MAX_STAGES) return false;
  int Ns = 1;
  for (int i = 0; i < nr; ++i) {
    StageInfo& si = out->st[i];
    si.R = rad[i];
    si.nb = L / rad[i];
    si.Ns = Ns;
    si.tstep = n_tab / (Ns * rad[i]);
    si.div_nb = FastDiv((uint32_t)si.nb);
    si.div_ns = FastDiv((uint32_t)Ns);
    Ns *= rad[i];
  }
  out->nst = nr;
  return true;
}

// Exported self-check of the integer division used by the kernels (host build
// of the same code); returns the number of mismatches.
extern "C" int64_t ur_selftest_fastdiv(void) {
  int64_t bad = 0;
  const uint32_t ds[] = {1, 2, 3, 5, 6, 7, 9, 10, 12, 14, 17, 31, 49, 96, 100, 125, 127, 129, 243, 257,
                         343, 385, 1000, 1025, 2049, 4097, 65537, 1000003};
  for (uint32_t d : ds) {
    FastDiv f(d);
    for (uint32_t x = 0; x < 70000; ++x)
      if (f.div(x) != x / d) ++bad;
    for (uint32_t x = (1u << 31) - 70000; x < (1u << 31); ++x)
      if (f.div(x) != x / d) ++bad;
  }
  return bad;
}

// Stage twiddles of the compile-time power-of-two transforms of length L = 2^lg
// with E = 8 or 16 values per thread: radix-E Stockham stages (the last one of a
// smaller radix when lg is not a multiple of log2 E).  Stage S >= 1 has NS = E^S
// butterfly classes k and radix R; its rows hold exp(-2 pi i r k / (NS R)) for
// r < R at row k (E slots, unused ones 0), so a butterfly reads its R - 1
// twiddles with at most E/2 16-byte loads.  Row blocks follow each other by
// stage.  Returns the number of float2 written (out may be NULL to count).
static size_t stage_twiddles(int lg, int E, float2* out) {
  const int le = E == 16 ? 4 : 3;
  const int nfull = lg / le, rem = lg % le, nst = nfull + (rem ? 1 : 0);
  size_t off = 0;
  long long ns = 1;
  for (int st = 0; st < nst; ++st) {
    const int R = st < nfull ? E : (1 << rem);
    if (st >= 1) {
      for (long long k = 0; k < ns; ++k)
        for (int r = 0; r < E; ++r) {
          float2 w = make_float2(0.f, 0.f);
          if (r < R) {
            const double a = 2.0 * M_PI * (double)(r * k) / (double)(ns * R);
            w = make_float2((float)cos(a), (float)(-sin(a)));
          }
          if (out) out[off + (size_t)k * E + r] = w;
        }
      off += (size_t)ns * E;
    }
    ns *= R;
  }
  return off;
}

// Butterfly check on the host: every compile-time radix of the row and column
// engines against a direct float64 DFT, forward and inverse, on seeded inputs.
// Returns the largest error relative to the input's L2 norm.
template <int R, bool INV>
static double dft_err(uint64_t& st) {
  float2 a[R];
  double re[R], im[R], nrm = 0.0;
  for (int p = 0; p < R; ++p) {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    re[p] = (double)(int32_t)(st >> 32) / 2147483648.0;
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    im[p] = (double)(int32_t)(st >> 32) / 2147483648.0;
    a[p] = make_float2((float)re[p], (float)im[p]);
    re[p] = a[p].x;
    im[p] = a[p].y;
    nrm += re[p] * re[p] + im[p] * im[p];
  }
  dft<R, INV>(a);
  const double sg = INV ? 1.0 : -1.0, tau = 6.283185307179586476925286766559;
  double err = 0.0;
  for (int k = 0; k < R; ++k) {
    double xr = 0.0, xi = 0.0;
    for (int p = 0; p < R; ++p) {
      const double ang = sg * tau * (double)((int64_t)p * k % R) / R;
      xr += re[p] * cos(ang) - im[p] * sin(ang);
      xi += re[p] * sin(ang) + im[p] * cos(ang);
    }
    err = fmax(err, hypot(a[k].x - xr, a[k].y - xi));
  }
  return err / sqrt(nrm);
}

template <int R>
static double dft_err_both(uint64_t& st) {
  double e = 0.0;
  for (int t = 0; t < 8; ++t) e = fmax(e, fmax(dft_err<R, false>(st), dft_err<R, true>(st)));
  return e;
}

extern "C" double ur_selftest_dft(void) {
  uint64_t st = 0x2303134350ULL;
  double e = 0.0;
  e = fmax(e, dft_err_both<2>(st));
  e = fmax(e, dft_err_both<3>(st));
  e = fmax(e, dft_err_both<4>(st));
  e = fmax(e, dft_err_both<5>(st));
  e = fmax(e, dft_err_both<7>(st));
  e = fmax(e, dft_err_both<8>(st));
  e = fmax(e, dft_err_both<16>(st));
  e = fmax(e, dft_err_both<32>(st));
  e = fmax(e, dft_err_both<6>(st));
  e = fmax(e, dft_err_both<9>(st));
  e = fmax(e, dft_err_both<10>(st));
  return e;
}

// ---------------------------------------------------------------------------
// Bin thresholds: t_j = min{s >= 0 : dq * sqrt(s) >= e_j} for j < B and
// t_B = min{s : dq * sqrt(s) > e_B}, in IEEE float64.  fl(dq * fl(sqrt(s))) is
// nondecreasing in s, so a binary search finds the exact crossing of the same
// float64 expression a per-voxel evaluation would use.
// ---------------------------------------------------------------------------
static inline double q_of(double dq, int64_t s) { return dq * sqrt((double)s); }

static int64_t first_s(double dq, double e, int64_t smax, bool strict) {
  int64_t lo = 0, hi = smax + 1;  // answer in [lo, hi]; hi = none
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    double q = q_of(dq, mid);
    bool ok = strict ? (q > e) : (q >= e);
    if (ok) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

extern "C" ur_status ur_bin_thresholds(int32_t n, double dx, const double* edges, int32_t nbins, int64_t* out) {
  UR_REQUIRE(n >= 2 && dx > 0 && edges && out && nbins >= 1, "ur_bin_thresholds: bad argument");
  const double dq = 2.0 * M_PI / ((double)n * dx);
  const int64_t smax = 3ll * (n / 2) * (n / 2);
  for (int j = 0; j <= nbins; ++j) out[j] = first_s(dq, edges[j], smax, j == nbins);
  return UR_OK;
}

static bool smooth_2357(int v) {
  if (v <= 0) return false;
  for (int p : {2, 3, 5, 7})
    while (v % p == 0) v /= p;
  return v == 1;
}

static void plan_free(ur_plan* p) {
  if (!p) return;
  if (p->tw) cudaFree(p->tw);
  if (p->stw) cudaFree(p->stw);
  if (p->thr) cudaFree(p->thr);
  if (p->geo) cudaFree(p->geo);
  if (p->d_sched) cudaFree(p->d_sched);
  if (p->binlut) cudaFree(p->binlut);
  if (p->bincoarse) cudaFree(p->bincoarse);
  if (p->zc_tw) cudaFree(p->zc_tw);
  if (p->vsinc) cudaFree(p->vsinc);
  if (p->zc_tiles) cudaFree(p->zc_tiles);
  free(p->thr_host);
  free(p);
}

template <typename K>
static int occupancy(K kern, int threads, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

// defined in ur_forward.cu: configures the kernels for a plan
ur_status ur_configure_kernels(ur_plan* p);

extern "C" ur_status ur_plan_create(const ur_grid_desc* g, const double* edges, int32_t nbins, ur_plan** out) {
  UR_REQUIRE(g && edges && out, "ur_plan_create: null argument");
  *out = nullptr;
  const int n = g->n;
  UR_REQUIRE(n >= 8 && n <= 4096 && n % 2 == 0 && smooth_2357(n / 2),
             "ur_plan_create: grid edge %d must be even, in [8, 4096], with N/2 a product of 2, 3, 5, 7", n);
  UR_REQUIRE(g->dx > 0 && isfinite(g->dx), "ur_plan_create: dx must be positive");
  UR_REQUIRE(g->ed_dtype == UR_F32 || g->ed_dtype == UR_F16, "ur_plan_create: ed_dtype must be UR_F32 or UR_F16");
  UR_REQUIRE(g->z0 >= 0 && g->nz >= 1 && g->z0 + g->nz <= n, "ur_plan_create: plane range [%d, %d) outside [0, %d)",
             g->z0, g->z0 + g->nz, n);
  UR_REQUIRE(nbins >= 1 && nbins <= 8192, "ur_plan_create: nbins %d outside [1, 8192]", nbins);
  for (int j = 0; j <= nbins; ++j) UR_REQUIRE(isfinite(edges[j]), "ur_plan_create: edge %d not finite", j);
  for (int j = 0; j < nbins; ++j) UR_REQUIRE(edges[j] < edges[j + 1], "ur_plan_create: edges must increase strictly");
  UR_TRY(ur_fault_point("plan_create"));

  ur_plan* p = (ur_plan*)calloc(1, sizeof(ur_plan));
  if (!p) {
    ur_set_error("ur_plan_create: out of host memory");
    return UR_ERR_OOM;
  }
  p->n = n;
  p->M = n / 2;
  p->H = n / 2 + 1;
  p->dx = g->dx;
  p->dq = 2.0 * M_PI / ((double)n * g->dx);
  p->ed_dtype = g->ed_dtype;
  p->z0 = g->z0;
  p->nz = g->nz;
  p->nbins = nbins;
  cudaGetDevice(&p->device);
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  if (p->num_sms <= 0) p->num_sms = 1;

  if (!ur_make_sched(n, n, &p->sched_n) || !ur_make_sched(p->M, n, &p->sched_m)) {
    plan_free(p);
    ur_set_error("ur_plan_create: no radix schedule for %d", n);
    return UR_ERR_INVALID;
  }

  // twiddles exp(-2 pi i t / n), float64 -> float32
  float2* tw_h = (float2*)malloc(sizeof(float2) * n);
  for (int t = 0; t < n; ++t) {
    double a = 2.0 * M_PI * (double)t / (double)n;
    tw_h[t] = make_float2((float)cos(a), (float)(-sin(a)));
  }
  // thresholds
  const int64_t smax = 3ll * (n / 2) * (n / 2);
  p->thr_host = (int64_t*)malloc(sizeof(int64_t) * (nbins + 1));
  int32_t* thr32 = (int32_t*)malloc(sizeof(int32_t) * (nbins + 1));
  for (int j = 0; j <= nbins; ++j) {
    int64_t t = first_s(p->dq, edges[j], smax, j == nbins);
    p->thr_host[j] = t;
    thr32[j] = (int32_t)(t > smax + 1 ? smax + 1 : t);
  }
  cudaError_t e1 = cudaMalloc(&p->tw, sizeof(float2) * n);
  cudaError_t e2 = cudaMalloc(&p->thr, sizeof(int32_t) * (nbins + 1));
  cudaError_t e3 = cudaMalloc(&p->geo, sizeof(double) * 2 * nbins);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    free(tw_h);
    free(thr32);
    plan_free(p);
    ur_set_error("ur_plan_create: device allocation of plan tables failed");
    return UR_ERR_OOM;
  }
  if (ur_fast_supported(n)) {
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    // columns (N points) run UR_FAST_COL_E(n) values per thread, rows (N/2 points) 8
    const int ecol = UR_FAST_COL_E(n);
    const size_t cn = stage_twiddles(lg, ecol, nullptr), cm = stage_twiddles(lg - 1, 8, nullptr);
    float2* st_h = (float2*)malloc(sizeof(float2) * (cn + cm + 1));
    stage_twiddles(lg, ecol, st_h);
    stage_twiddles(lg - 1, 8, st_h + cn);
    p->stw_m_off = (int)cn;
    const cudaError_t ea = cudaMalloc(&p->stw, sizeof(float2) * (cn + cm + 1));
    const cudaError_t eb = ea == cudaSuccess ? cudaMemcpy(p->stw, st_h, sizeof(float2) * (cn + cm + 1),
                                                          cudaMemcpyHostToDevice) : ea;
    free(st_h);
    if (eb != cudaSuccess) {
      free(tw_h);
      free(thr32);
      plan_free(p);
      ur_set_error("ur_plan_create: stage twiddle table: %s", cudaGetErrorString(eb));
      return ea != cudaSuccess ? UR_ERR_OOM : UR_ERR_CUDA;
    }
  }
  cudaError_t e4 = cudaMemcpy(p->tw, tw_h, sizeof(float2) * n, cudaMemcpyHostToDevice);
  cudaError_t e5 = cudaMemcpy(p->thr, thr32, sizeof(int32_t) * (nbins + 1), cudaMemcpyHostToDevice);
  free(tw_h);
  free(thr32);
  if (e4 != cudaSuccess || e5 != cudaSuccess) {
    plan_free(p);
    ur_set_error("ur_plan_create: copy of plan tables failed: %s", cudaGetErrorString(e4 != cudaSuccess ? e4 : e5));
    return UR_ERR_CUDA;
  }
  ur_status st = ur_configure_kernels(p);
  if (st != UR_OK) {
    plan_free(p);
    return st;
  }
  // data-independent bin geometry (count and sum |Q| per bin)
  st = ur_launch_geometry(p, 0);
  if (st == UR_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      ur_set_error("ur_plan_create: bin geometry kernel failed: %s", cudaGetErrorString(e));
      st = UR_ERR_CUDA;
    }
  }
  if (st == UR_OK) st = ur_zcol_prepare(p);
  if (st != UR_OK) {
    plan_free(p);
    return st;
  }
  *out = p;
  return UR_OK;
}

extern "C" ur_status ur_plan_set_voxel_sinc(ur_plan* p, int32_t on) {
  UR_REQUIRE(p, "ur_plan_set_voxel_sinc: null plan");
  if (!on) {
    if (p->vsinc) cudaFree(p->vsinc);
    p->vsinc = nullptr;
    return UR_OK;
  }
  if (p->vsinc) return UR_OK;
  const int M = p->M;
  float* h = (float*)malloc(sizeof(float) * (M + 1));
  for (int m = 0; m <= M; ++m) {
    const double a = M_PI * (double)m / (double)p->n;
    const double sn = m == 0 ? 1.0 : sin(a) / a;
    h[m] = (float)(sn * sn);
  }
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(float) * (M + 1));
  if (e == cudaSuccess) e = cudaMemcpy(d, h, sizeof(float) * (M + 1), cudaMemcpyHostToDevice);
  free(h);
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    ur_set_error("ur_plan_set_voxel_sinc: %s", cudaGetErrorString(e));
    return UR_ERR_OOM;
  }
  p->vsinc = d;
  return UR_OK;
}

extern "C" int32_t ur_plan_voxel_sinc(const ur_plan* p) { return (p && p->vsinc) ? 1 : 0; }

extern "C" ur_status ur_plan_destroy(ur_plan* p) {
  plan_free(p);
  return UR_OK;
}

extern "C" ur_status ur_plan_thresholds(const ur_plan* p, int64_t* out) {
  UR_REQUIRE(p && out, "ur_plan_thresholds: null argument");
  memcpy(out, p->thr_host, sizeof(int64_t) * (p->nbins + 1));
  return UR_OK;
}

extern "C" size_t ur_workspace_size(const ur_plan* p, int32_t what) {
  if (!p) return 0;
  size_t b = 0;
  if (what & (UR_WS_FORWARD | UR_WS_BACKWARD)) b += ur_align_up(p->ws_inter, 256);
  if (what & UR_WS_BACKWARD)
    b += ur_align_up(p->ws_inv, 256) + ur_align_up(p->ws_sigma, 256) + ur_align_up(p->ws_chunk, 256);
  if (what & UR_WS_HOST_SLABS) b += 2 * ur_align_up(p->ws_slab, 256);
  if (what & UR_WS_ADJ_SLABS) {
    // fixed layout after the forward intermediate: [host staging slabs][Y slab][sigma][two dL/dm slabs]
    const size_t S = (size_t)p->adj_slab_planes;
    if (!(what & UR_WS_HOST_SLABS)) b += 2 * ur_align_up(p->ws_slab, 256);
    b += ur_align_up(S * p->n * p->H * sizeof(float2), 256) + ur_align_up(p->ws_sigma, 256) +
         2 * ur_align_up((size_t)ur_adj_dm_planes(p) * p->n * p->n * sizeof(float), 256);
  }
  return b;
}

// ---------------------------------------------------------------------------
// Merge (Sec. 2.5 last paragraph; Fig. 2 caption; Sec. 2.7 for the
// uncertainty-weighted combination): one thread per output bin.
// ---------------------------------------------------------------------------
#define UR_MAX_LEVELS 8
struct MergeArgs {
  const double* bins[UR_MAX_LEVELS];  // in window order (coarsest level first)
  double scale[UR_MAX_LEVELS];        // N^6
  double qlo[UR_MAX_LEVELS];          // window lower edge, in window order
  double qhi[UR_MAX_LEVELS];          // level limit pi/dx
  int order[UR_MAX_LEVELS];           // caller's level index of the t-th window
  int pos[UR_MAX_LEVELS];             // window position of the caller's level i
  int nlev, mode;
};

// Q_max/2 artefact limit of a level (Fig. 2 caption) with Q_max = 2 pi/dx the sampling frequency
extern "C" double ur_level_qmax(double dx) { return (dx > 0 && isfinite(dx)) ? M_PI / dx : 0.0; }

__global__ void k_merge(MergeArgs a, const double* __restrict__ edges, int nb, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const double c = sqrt(edges[j] * edges[j + 1]);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double mean = nan, sem = nan, cnt = 0.0, q = nan, src = -1.0;
  bool done = false;
  if (a.mode == UR_MERGE_INVVAR) {
    // every level trusted at the bin centre with voxels and a usable SEM, weight 1/SEM^2,
    // accumulated in the caller's level order
    double sw = 0.0, swm = 0.0, sn = 0.0, sq = 0.0, best_w = -1.0;
    int best = -1;
    for (int i = 0; i < a.nlev; ++i) {
      const int t = a.pos[i];
      const double* b = a.bins[t];
      const double n = b[UR_BIN_COUNT * nb + j];
      if (c > a.qhi[t] || !(n > 0)) continue;
      const double s_abs = b[UR_BIN_SEM * nb + j] * a.scale[t];
      if (!(isfinite(s_abs) && s_abs > 0)) continue;
      const double w = 1.0 / (s_abs * s_abs);
      sw += w;
      swm += w * (b[UR_BIN_MEAN * nb + j] * a.scale[t]);
      sn += n;
      sq += b[UR_BIN_SUM_Q * nb + j];
      if (w > best_w) {
        best_w = w;
        best = i;
      }
    }
    if (best >= 0) {
      mean = swm / sw;
      sem = 1.0 / sqrt(sw);
      cnt = sn;
      q = sq / sn;
      src = (double)best;
      done = true;
    }
  }
  if (!done) {
    int pick = -1;
    for (int t = 0; t < a.nlev; ++t) {
      const bool last = t == a.nlev - 1;
      if ((a.qlo[t] <= c && c < a.qhi[t]) || (last && c == a.qhi[t])) {
        pick = t;
        break;
      }
    }
    if (pick >= 0) {
      const double* b = a.bins[pick];
      const double n = b[UR_BIN_COUNT * nb + j];
      if (n > 0) {
        const double s = a.scale[pick];
        mean = b[UR_BIN_MEAN * nb + j] * s;
        sem = b[UR_BIN_SEM * nb + j] * s;
        cnt = n;
        q = b[UR_BIN_SUM_Q * nb + j] / n;
        src = (double)a.order[pick];
      }
    }
  }
  out[0 * nb + j] = mean;
  out[1 * nb + j] = sem;
  out[2 * nb + j] = cnt;
  out[3 * nb + j] = q;
  out[4 * nb + j] = src;
}

extern "C" ur_status ur_merge(int32_t nlev, const double* const* level_bins, const int32_t* level_n,
                              const double* level_dx, const double* edges, int32_t nbins, int32_t mode, double* out,
                              void* stream) {
  UR_REQUIRE(nlev >= 1 && nlev <= UR_MAX_LEVELS, "ur_merge: nlev %d outside [1, %d]", nlev, UR_MAX_LEVELS);
  UR_REQUIRE(level_bins && level_n && level_dx && edges && out, "ur_merge: null argument");
  UR_REQUIRE(nbins >= 1, "ur_merge: nbins must be positive");
  UR_REQUIRE(mode == UR_MERGE_WINDOWS || mode == UR_MERGE_INVVAR, "ur_merge: unknown mode %d", mode);
  MergeArgs a;
  memset(&a, 0, sizeof a);
  a.nlev = nlev;
  a.mode = mode;
  int idx[UR_MAX_LEVELS];
  double qmax[UR_MAX_LEVELS];
  for (int i = 0; i < nlev; ++i) {
    UR_REQUIRE(level_bins[i], "ur_merge: level %d has no bins", i);
    UR_REQUIRE(level_n[i] > 0 && level_dx[i] > 0 && isfinite(level_dx[i]), "ur_merge: level %d has a bad size or dx", i);
    qmax[i] = ur_level_qmax(level_dx[i]);
    idx[i] = i;
  }
  // windows ordered by their upper limit (coarsest level first); stable
  for (int i = 1; i < nlev; ++i)
    for (int k = i; k > 0 && qmax[idx[k]] < qmax[idx[k - 1]]; --k) {
      int t = idx[k];
      idx[k] = idx[k - 1];
      idx[k - 1] = t;
    }
  double lo = 0.0;
  for (int t = 0; t < nlev; ++t) {
    const int i = idx[t];
    a.bins[t] = level_bins[i];
    double nn = (double)level_n[i];
    a.scale[t] = nn * nn * nn * nn * nn * nn;
    a.qlo[t] = lo;
    a.qhi[t] = qmax[i];
    a.order[t] = i;
    a.pos[i] = t;
    lo = qmax[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_merge<<<(nbins + 127) / 128, 128, 0, s>>>(a, edges, nbins, out);
  UR_LAUNCH_CHECK("k_merge");
  return UR_OK;
}

// ---------------------------------------------------------------------------
// Polydisperse ensemble (Sec. 3: volume-weighted single-particle simulations summed
// into one curve): one thread per bin.  The item tables travel as kernel parameters
// (by value, so the launch can be captured in a CUDA graph).
// ---------------------------------------------------------------------------
#define UR_MAX_ENSEMBLE 512
struct EnsembleArgs {
  const double* bins[UR_MAX_ENSEMBLE];
  double* grad[UR_MAX_ENSEMBLE];
  double scale[UR_MAX_ENSEMBLE];  // w_i N_i^6
  int count;
};

__device__ __forceinline__ bool ens_valid(const EnsembleArgs& a, int nb, int j) {
  for (int i = 0; i < a.count; ++i)
    if (a.scale[i] != 0.0 && !(a.bins[i][UR_BIN_COUNT * nb + j] > 0)) return false;
  return true;
}

__global__ void k_ensemble(const __grid_constant__ EnsembleArgs a, int nb, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double mean = nan, sem = nan, cnt = 0.0, q = nan;
  if (ens_valid(a, nb, j)) {
    double s = 0.0, v = 0.0, c = 0.0, cq = 0.0;
    for (int i = 0; i < a.count; ++i) {
      const double sc = a.scale[i];
      if (sc == 0.0) continue;
      const double* b = a.bins[i];
      s += sc * b[UR_BIN_MEAN * nb + j];
      const double e = sc * b[UR_BIN_SEM * nb + j];
      v += e * e;
      c += b[UR_BIN_COUNT * nb + j];
      cq += b[UR_BIN_SUM_Q * nb + j];
    }
    mean = s;
    sem = sqrt(v);
    cnt = c;
    q = cq / c;
  }
  out[0 * nb + j] = mean;
  out[1 * nb + j] = sem;
  out[2 * nb + j] = cnt;
  out[3 * nb + j] = q;
}

__global__ void k_ensemble_grad(const __grid_constant__ EnsembleArgs a, int nb, const double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const bool ok = ens_valid(a, nb, j) && isfinite(g[j]);
  for (int i = 0; i < a.count; ++i) a.grad[i][j] = ok ? a.scale[i] * g[j] : 0.0;
}

static ur_status ensemble_args(int32_t count, const double* const* item_bins, const int32_t* item_n,
                               const double* weights, double* const* item_grad, EnsembleArgs* a) {
  UR_REQUIRE(count >= 1 && count <= UR_MAX_ENSEMBLE, "ensemble: %d items (1..%d)", count, UR_MAX_ENSEMBLE);
  UR_REQUIRE(item_bins && item_n && weights, "ensemble: null argument");
  memset(a, 0, sizeof *a);
  a->count = count;
  for (int i = 0; i < count; ++i) {
    UR_REQUIRE(item_bins[i] && item_n[i] > 0 && isfinite(weights[i]),
               "ensemble: item %d has no bins, a bad size or a non-finite weight", i);
    UR_REQUIRE(!item_grad || item_grad[i], "ensemble: item %d has no gradient output", i);
    a->bins[i] = item_bins[i];
    a->grad[i] = item_grad ? item_grad[i] : nullptr;
    const double nn = (double)item_n[i];
    a->scale[i] = weights[i] * nn * nn * nn * nn * nn * nn;
  }
  return UR_OK;
}

extern "C" ur_status ur_ensemble(int32_t count, const double* const* item_bins, const int32_t* item_n,
                                 const double* weights, int32_t nbins, double* out, void* stream) {
  UR_REQUIRE(nbins >= 1 && out, "ur_ensemble: bad argument");
  EnsembleArgs* a = (EnsembleArgs*)malloc(sizeof(EnsembleArgs));
  if (!a) {
    ur_set_error("ur_ensemble: out of host memory");
    return UR_ERR_OOM;
  }
  ur_status st = ensemble_args(count, item_bins, item_n, weights, nullptr, a);
  if (st == UR_OK) {
    k_ensemble<<<(nbins + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*a, nbins, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ur_set_error("launch of k_ensemble failed: %s", cudaGetErrorString(e));
      st = UR_ERR_CUDA;
    }
  }
  free(a);
  return st;
}

extern "C" ur_status ur_ensemble_backward(int32_t count, const double* const* item_bins, const int32_t* item_n,
                                          const double* weights, int32_t nbins, const double* dl_dens,
                                          double* const* item_dl_dmean, void* stream) {
  UR_REQUIRE(nbins >= 1 && dl_dens && item_dl_dmean, "ur_ensemble_backward: bad argument");
  EnsembleArgs* a = (EnsembleArgs*)malloc(sizeof(EnsembleArgs));
  if (!a) {
    ur_set_error("ur_ensemble_backward: out of host memory");
    return UR_ERR_OOM;
  }
  ur_status st = ensemble_args(count, item_bins, item_n, weights, item_dl_dmean, a);
  if (st == UR_OK) {
    k_ensemble_grad<<<(nbins + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*a, nbins, dl_dens);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ur_set_error("launch of k_ensemble_grad failed: %s", cudaGetErrorString(e));
      st = UR_ERR_CUDA;
    }
  }
  free(a);
  return st;
}
