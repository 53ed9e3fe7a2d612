// Batched particles of uneven grid sizes (the paper's polydisperse ensembles,
// Sec. 3: many particle simulations summed or fitted together).
//
// A ur_batch is built once from per-particle items (plan, shape, buffers).  It
// holds device tables that give every kernel block its (particle, tile): each
// pass over the whole batch is then a single launch of a generic kernel whose
// blocks read their particle's arguments from the table, so the forward and
// the adjoint of the whole batch are five launches each, with no host work
// between them (capturable in one CUDA graph).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ur_fast.cuh"

struct ur_batch {
  int count;
  int maxnb;
  void* dev;  // one allocation holding every table
  BatchZeroItem* zero_bins;
  BatchRowsItem* rows;
  long long* rows_start;
  ColArgs* coly;
  long long* coly_start;
  ColArgs* zbin;
  long long* zbin_start;
  BatchFinItem* fin;
  BatchSigmaItem* sig;
  ColArgs* zadj;
  long long* zadj_start;
  ColArgs* yinv;
  long long* yinv_start;
  BatchZeroItem* zero_cell;
  BatchGradItem* grad;
  long long* grad_start;
  long long nb_rows, nb_coly, nb_zbin, nb_zadj, nb_yinv, nb_grad;
  size_t smem_rows, smem_cols, smem_zbin, smem_grad;
  int has_backward;
};

extern "C" ur_status ur_plan_set_tiles(ur_plan* p, int32_t rows_per_block, int32_t cols_per_block) {
  UR_REQUIRE(p, "ur_plan_set_tiles: null plan");
  if (rows_per_block > 0) {
    UR_REQUIRE((long long)rows_per_block * p->M <= (long long)UR_EMAX * p->row_threads,
               "ur_plan_set_tiles: %d rows of %d exceed a block's %d elements", rows_per_block, p->M,
               UR_EMAX * p->row_threads);
    p->row_rb = rows_per_block;
    p->row_smem = (size_t)rows_per_block * p->M * sizeof(float2);
  }
  if (cols_per_block > 0) {
    UR_REQUIRE((long long)cols_per_block * p->n <= (long long)UR_EMAX * p->col_threads,
               "ur_plan_set_tiles: %d columns of %d exceed a block's %d elements", cols_per_block, p->n,
               UR_EMAX * p->col_threads);
    p->col_tx = cols_per_block;
    p->col_smem = ur_align_up((size_t)cols_per_block * (p->n + 1) * sizeof(float2), 16) +
                  ur_align_up((size_t)(p->nbins + 1) * 4, 16);
    p->colbin_smem = p->col_smem + (size_t)p->nbins * 16;
    p->zbin_grid = (int)(((long long)p->n * p->H + cols_per_block - 1) / cols_per_block);
  }
  return UR_OK;
}

extern "C" ur_status ur_plan_get_tiles(const ur_plan* p, int32_t* rows_per_block, int32_t* cols_per_block) {
  UR_REQUIRE(p && rows_per_block && cols_per_block, "ur_plan_get_tiles: null argument");
  *rows_per_block = p->row_rb;
  *cols_per_block = p->col_tx;
  return UR_OK;
}

template <typename T>
static size_t table_bytes(int count) {
  return ur_align_up(sizeof(T) * (size_t)count, 256);
}

extern "C" ur_status ur_batch_create(int32_t count, const ur_batch_item* items, ur_batch** out) {
  UR_REQUIRE(out && items && count >= 1 && count <= 65535, "ur_batch_create: need 1..65535 items");
  *out = nullptr;
  std::vector<BatchZeroItem> zb(count), zc(count);
  std::vector<BatchRowsItem> rows(count);
  std::vector<ColArgs> coly(count), zbin(count), zadj(count), yinv(count);
  std::vector<BatchFinItem> fin(count);
  std::vector<BatchSigmaItem> sig(count);
  std::vector<BatchGradItem> grad(count);
  std::vector<long long> s_rows(count + 1), s_coly(count + 1), s_zbin(count + 1), s_zadj(count + 1), s_yinv(count + 1),
      s_grad(count + 1);
  size_t smem_rows = 0, smem_cols = 0, smem_zbin = 0, smem_grad = 0;
  int maxnb = 0, has_bwd = 1;
  for (int i = 0; i < count; ++i) {
    const ur_batch_item& it = items[i];
    const ur_plan* p = it.plan;
    UR_REQUIRE(p && it.cell && it.bins && it.ws, "ur_batch_create: item %d has a null plan, cell, bins or ws", i);
    UR_REQUIRE(it.ucell >= 1 && (long long)it.ucell * it.ucell <= 65535, "ur_batch_create: item %d cell edge", i);
    UR_REQUIRE(it.shape.kind >= UR_SHAPE_SPHERE && it.shape.kind <= UR_SHAPE_WEIGHTS, "ur_batch_create: item %d shape", i);
    UR_REQUIRE(it.shape.kind != UR_SHAPE_WEIGHTS || it.weights, "ur_batch_create: item %d needs weights", i);
    UR_REQUIRE(it.origin[0] >= 0 && it.origin[1] >= 0 && it.origin[2] >= 0, "ur_batch_create: item %d origin must be >= 0",
               i);
    UR_REQUIRE(((uintptr_t)it.ws % 256) == 0, "ur_batch_create: item %d workspace misaligned", i);
    const bool bwd = it.dl_dmean && it.dl_dcell;
    has_bwd &= bwd ? 1 : 0;
    if (bwd && p->vsinc) {
      ur_set_error("ur_batch_create: item %d: the adjoint of the voxel-sinc corrected binning is not built", i);
      return UR_ERR_UNSUPPORTED;
    }
    const size_t need = ur_workspace_size(p, bwd ? (UR_WS_FORWARD | UR_WS_BACKWARD) : UR_WS_FORWARD);
    UR_REQUIRE(it.ws_bytes >= need, "ur_batch_create: item %d workspace %zu < %zu bytes", i, it.ws_bytes, need);
    const int n = p->n, H = p->H, M = p->M, nb = p->nbins;
    if (nb > maxnb) maxnb = nb;
    const double n3 = (double)n * n * n;
    float2* X = (float2*)it.ws;
    float2* Y = (float2*)((char*)it.ws + ur_align_up(p->ws_inter, 256));
    float* sigma = (float*)((char*)Y + ur_align_up(p->ws_inv, 256));
    const ShapeArgs sh = ur_shape_args(&it.shape);
    const float* weights = it.shape.kind == UR_SHAPE_WEIGHTS ? it.weights : nullptr;
    // forward: rows with the density generated in the kernel
    BatchRowsItem& r = rows[i];
    memset(&r, 0, sizeof r);
    r.ra.X = X;
    r.ra.nrows = (long long)p->nz * n;
    r.ra.z0 = p->z0;
    r.ra.cell = it.cell;
    r.ra.ucell = it.ucell;
    r.ra.ox = it.origin[0];
    r.ra.oy = it.origin[1];
    r.ra.oz = it.origin[2];
    r.ra.sh = sh;
    r.ra.weights = weights;
    r.ra.tw = p->tw;
    r.N = n;
    r.RB = p->row_rb;
    r.nst = p->sched_m.nst;
    r.gen = 1;
    r.sched = p->d_sched + UR_MAX_STAGES;
    s_rows[i + 1] = s_rows[i] + (r.ra.nrows + r.RB - 1) / r.RB;
    smem_rows = std::max(smem_rows, (size_t)r.RB * M * sizeof(float2));
    // y columns, in place
    ColArgs a = ur_col_args(p);
    a.src = X;
    a.dst = X;
    a.ncols = (long long)p->nz * H;
    a.A = (long long)n * H;
    a.S = H;
    a.Ad = a.A;
    a.Sd = a.S;
    a.nload = n;
    a.zoff = 0;
    a.nbins = 0;
    coly[i] = a;
    s_coly[i + 1] = s_coly[i] + (a.ncols + a.TX - 1) / a.TX;
    smem_cols = std::max(smem_cols, p->col_smem);
    // z columns + bins
    ColArgs zb_ = ur_col_args(p);
    zb_.src = X;
    zb_.ncols = (long long)n * H;
    zb_.A = H;
    zb_.S = (long long)n * H;
    zb_.nload = p->nz;
    zb_.zoff = p->z0;
    zb_.iscale = (float)(1.0 / n3);
    zb_.gsum = it.bins + UR_BIN_SUM_I * nb;
    zb_.gsum2 = it.bins + UR_BIN_SUM_I2 * nb;
    zbin[i] = zb_;
    s_zbin[i + 1] = s_zbin[i] + (zb_.ncols + zb_.TX - 1) / zb_.TX;
    smem_zbin = std::max(smem_zbin, p->colbin_smem);
    zb[i].ptr = it.bins;
    zb[i].bytes = sizeof(double) * UR_BIN_FIELDS * nb;
    fin[i].bins = it.bins;
    fin[i].geo = p->geo;
    fin[i].nb = nb;
    fin[i].inv_n3 = 1.0 / n3;
    // adjoint
    sig[i].g = it.dl_dmean;
    sig[i].bins = it.bins;
    sig[i].nb = nb;
    sig[i].n3 = n3;
    sig[i].sigma = sigma;
    ColArgs za = ur_col_args(p);
    za.src = X;
    za.dst = Y;
    za.ncols = (long long)n * H;
    za.A = H;
    za.S = (long long)n * H;
    za.Ad = H;
    za.Sd = (long long)n * H;
    za.nload = p->nz;
    za.zoff = p->z0;
    za.sigma = sigma;
    zadj[i] = za;
    s_zadj[i + 1] = s_zadj[i] + (za.ncols + za.TX - 1) / za.TX;
    ColArgs yi = ur_col_args(p);
    yi.src = Y;
    yi.dst = Y;
    yi.ncols = (long long)n * H;
    yi.A = (long long)n * H;
    yi.S = H;
    yi.Ad = yi.A;
    yi.Sd = yi.S;
    yi.nload = n;
    yi.zoff = 0;
    yi.nbins = 0;
    yinv[i] = yi;
    s_yinv[i + 1] = s_yinv[i] + (yi.ncols + yi.TX - 1) / yi.TX;
    zc[i].ptr = it.dl_dcell;
    zc[i].bytes = bwd ? sizeof(float) * (size_t)it.ucell * it.ucell * it.ucell : 0;
    BatchGradItem& g = grad[i];
    memset(&g, 0, sizeof g);
    g.g.Y = Y;
    g.g.N = n;
    g.g.RB = p->row_rb;
    g.g.nst = p->sched_m.nst;
    g.g.sched = p->d_sched + UR_MAX_STAGES;
    g.g.tw = p->tw;
    g.g.cell = it.cell;
    g.g.U = it.ucell;
    g.g.ox = it.origin[0];
    g.g.oy = it.origin[1];
    g.g.oz = it.origin[2];
    g.g.sh = sh;
    g.g.weights = weights;
    g.g.inv_n3 = (float)(1.0 / n3);
    g.g.dl_dmask = it.dl_dmask;
    g.g.dl_dcell = it.dl_dcell;
    const int rpg = ((n + it.ucell - 1) / it.ucell) * ((n + it.ucell - 1) / it.ucell);
    g.gx = (rpg + g.g.RB - 1) / g.g.RB;
    s_grad[i + 1] = s_grad[i] + (long long)g.gx * it.ucell * it.ucell;
    smem_grad = std::max(smem_grad, ur_align_up((size_t)g.g.RB * H * sizeof(float2), 16) + (size_t)it.ucell * 4);
  }
  UR_REQUIRE(smem_grad <= 227 * 1024 && smem_zbin <= 227 * 1024, "ur_batch_create: shared memory per block too large");

  ur_batch* b = (ur_batch*)calloc(1, sizeof(ur_batch));
  if (!b) {
    ur_set_error("ur_batch_create: out of host memory");
    return UR_ERR_OOM;
  }
  b->count = count;
  b->maxnb = maxnb;
  b->has_backward = has_bwd;
  const size_t o_zb = 0;
  const size_t o_rows = o_zb + table_bytes<BatchZeroItem>(count);
  const size_t o_rs = o_rows + table_bytes<BatchRowsItem>(count);
  const size_t o_coly = o_rs + table_bytes<long long>(count + 1);
  const size_t o_cs = o_coly + table_bytes<ColArgs>(count);
  const size_t o_zbin = o_cs + table_bytes<long long>(count + 1);
  const size_t o_zs = o_zbin + table_bytes<ColArgs>(count);
  const size_t o_fin = o_zs + table_bytes<long long>(count + 1);
  const size_t o_sig = o_fin + table_bytes<BatchFinItem>(count);
  const size_t o_zadj = o_sig + table_bytes<BatchSigmaItem>(count);
  const size_t o_zas = o_zadj + table_bytes<ColArgs>(count);
  const size_t o_yinv = o_zas + table_bytes<long long>(count + 1);
  const size_t o_yis = o_yinv + table_bytes<ColArgs>(count);
  const size_t o_zc = o_yis + table_bytes<long long>(count + 1);
  const size_t o_grad = o_zc + table_bytes<BatchZeroItem>(count);
  const size_t o_gs = o_grad + table_bytes<BatchGradItem>(count);
  const size_t total = o_gs + table_bytes<long long>(count + 1);
  if (cudaMalloc(&b->dev, total) != cudaSuccess) {
    free(b);
    ur_set_error("ur_batch_create: device allocation of %zu bytes of tables failed", total);
    return UR_ERR_OOM;
  }
  std::vector<char> host(total, 0);
  auto put = [&](size_t off, const void* src, size_t bytes) { memcpy(host.data() + off, src, bytes); };
  put(o_zb, zb.data(), sizeof(BatchZeroItem) * count);
  put(o_rows, rows.data(), sizeof(BatchRowsItem) * count);
  put(o_rs, s_rows.data(), sizeof(long long) * (count + 1));
  put(o_coly, coly.data(), sizeof(ColArgs) * count);
  put(o_cs, s_coly.data(), sizeof(long long) * (count + 1));
  put(o_zbin, zbin.data(), sizeof(ColArgs) * count);
  put(o_zs, s_zbin.data(), sizeof(long long) * (count + 1));
  put(o_fin, fin.data(), sizeof(BatchFinItem) * count);
  put(o_sig, sig.data(), sizeof(BatchSigmaItem) * count);
  put(o_zadj, zadj.data(), sizeof(ColArgs) * count);
  put(o_zas, s_zadj.data(), sizeof(long long) * (count + 1));
  put(o_yinv, yinv.data(), sizeof(ColArgs) * count);
  put(o_yis, s_yinv.data(), sizeof(long long) * (count + 1));
  put(o_zc, zc.data(), sizeof(BatchZeroItem) * count);
  put(o_grad, grad.data(), sizeof(BatchGradItem) * count);
  put(o_gs, s_grad.data(), sizeof(long long) * (count + 1));
  if (cudaMemcpy(b->dev, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(b->dev);
    free(b);
    ur_set_error("ur_batch_create: upload of the batch tables failed");
    return UR_ERR_CUDA;
  }
  char* d = (char*)b->dev;
  b->zero_bins = (BatchZeroItem*)(d + o_zb);
  b->rows = (BatchRowsItem*)(d + o_rows);
  b->rows_start = (long long*)(d + o_rs);
  b->coly = (ColArgs*)(d + o_coly);
  b->coly_start = (long long*)(d + o_cs);
  b->zbin = (ColArgs*)(d + o_zbin);
  b->zbin_start = (long long*)(d + o_zs);
  b->fin = (BatchFinItem*)(d + o_fin);
  b->sig = (BatchSigmaItem*)(d + o_sig);
  b->zadj = (ColArgs*)(d + o_zadj);
  b->zadj_start = (long long*)(d + o_zas);
  b->yinv = (ColArgs*)(d + o_yinv);
  b->yinv_start = (long long*)(d + o_yis);
  b->zero_cell = (BatchZeroItem*)(d + o_zc);
  b->grad = (BatchGradItem*)(d + o_grad);
  b->grad_start = (long long*)(d + o_gs);
  b->nb_rows = s_rows[count];
  b->nb_coly = s_coly[count];
  b->nb_zbin = s_zbin[count];
  b->nb_zadj = s_zadj[count];
  b->nb_yinv = s_yinv[count];
  b->nb_grad = s_grad[count];
  b->smem_rows = smem_rows;
  b->smem_cols = smem_cols;
  b->smem_zbin = smem_zbin;
  b->smem_grad = smem_grad;
  *out = b;
  return UR_OK;
}

extern "C" ur_status ur_batch_destroy(ur_batch* b) {
  if (b) {
    if (b->dev) cudaFree(b->dev);
    free(b);
  }
  return UR_OK;
}

extern "C" ur_status ur_batch_forward(const ur_batch* b, void* stream) {
  UR_REQUIRE(b, "ur_batch_forward: null batch");
  cudaStream_t s = (cudaStream_t)stream;
  ur_timing_begin("batch_zero_bins", s);
  UR_TRY(ur_batch_launch_zero(b->zero_bins, b->count, s));
  ur_timing_end(s);
  ur_timing_begin("batch_rows", s);
  UR_TRY(ur_batch_launch_rows(b->rows, b->rows_start, b->count, b->nb_rows, b->smem_rows, s));
  ur_timing_end(s);
  ur_timing_begin("batch_cols_y", s);
  UR_TRY(ur_batch_launch_cols(COL_Y, false, b->coly, b->coly_start, b->count, b->nb_coly, b->smem_cols, s));
  ur_timing_end(s);
  ur_timing_begin("batch_cols_z_bin", s);
  UR_TRY(ur_batch_launch_cols(COL_ZBIN, false, b->zbin, b->zbin_start, b->count, b->nb_zbin, b->smem_zbin, s));
  ur_timing_end(s);
  ur_timing_begin("batch_finalize", s);
  UR_TRY(ur_batch_launch_finalize(b->fin, b->count, b->maxnb, s));
  ur_timing_end(s);
  return UR_OK;
}

extern "C" ur_status ur_batch_backward(const ur_batch* b, void* stream) {
  UR_REQUIRE(b, "ur_batch_backward: null batch");
  UR_REQUIRE(b->has_backward, "ur_batch_backward: the batch items carry no dl_dmean/dl_dcell");
  cudaStream_t s = (cudaStream_t)stream;
  ur_timing_begin("batch_sigma", s);
  UR_TRY(ur_batch_launch_sigma(b->sig, b->count, b->maxnb, s));
  ur_timing_end(s);
  ur_timing_begin("batch_adj_cols_z", s);
  UR_TRY(ur_batch_launch_cols(COL_ZADJ, false, b->zadj, b->zadj_start, b->count, b->nb_zadj, b->smem_cols, s));
  ur_timing_end(s);
  ur_timing_begin("batch_adj_cols_y", s);
  UR_TRY(ur_batch_launch_cols(COL_Y, true, b->yinv, b->yinv_start, b->count, b->nb_yinv, b->smem_cols, s));
  ur_timing_end(s);
  ur_timing_begin("batch_zero_cell", s);
  UR_TRY(ur_batch_launch_zero(b->zero_cell, b->count, s));
  ur_timing_end(s);
  ur_timing_begin("batch_adj_rows_grad", s);
  UR_TRY(ur_batch_launch_grad(b->grad, b->grad_start, b->count, b->nb_grad, b->smem_grad, s));
  ur_timing_end(s);
  return UR_OK;
}
