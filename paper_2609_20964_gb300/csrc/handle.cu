// C ABI entry points: handle lifecycle, argument validation, workspace layout
// and the order of the stages of a forward / query / backward call.
#include <math.h>
#include <string.h>

#include <new>

#include "wgeo_internal.cuh"

namespace wgeo {
int sh_valid_K(int K);
}

using namespace wgeo;

namespace {

constexpr size_t kAlign = 256;

struct Layout {
  size_t total = 0;
  size_t off_b32, off_chi32, off_chi64, off_r32, off_e32, off_phi, off_ctri, off_dphi, off_dchi64,
      off_lam64, off_lam32, off_levels, off_dct, off_pcell, off_pfrac, off_pnrm, off_srec, off_tile_count,
      off_tile_off, off_tile_cursor, off_brick_count, off_brick_off, off_leaf_off, off_leaf_cnt, off_tris, off_tris_lo, off_tris_s, off_cell_pyr, off_pyr, off_pyr_sums, off_pyr_rth, off_partials,
      off_scan, off_state, off_dp_cell, off_dp_count, off_dp_off, off_dp_cursor, off_dp_scan, off_dp_tmp,
      off_dp_sorted, off_dp_key, off_dp_gbox, off_or_scal;
  size_t n_partials, n_scan, n_dp_scan;
  int64_t dp_cap, dp_points;
  int64_t cap;
};

size_t take(size_t& cur, size_t bytes) {
  cur = (cur + kAlign - 1) / kAlign * kAlign;
  const size_t o = cur;
  cur += bytes;
  return o;
}

bool valid_res(int res) { return res >= 4 && res <= kMaxRes && coarsest_size(res) <= 16; }

Layout make_layout(int R, int64_t P, const wgeo_options& opt) {
  Layout L;
  const size_t N = (size_t)R * R * R;
  const bool keep = opt.keep_for_backward != 0;
  size_t c = 0;
  L.off_b32 = take(c, 4 * N);
  L.off_chi32 = take(c, 4 * N);
  L.off_chi64 = take(c, 16 * N);                       // two float-float buffers
  L.off_r32 = take(c, 4 * N);
  L.off_e32 = take(c, 4 * N);
  L.off_phi = take(c, 4 * N);
  L.off_ctri = take(c, keep ? 4 * N : 0);
  L.off_dphi = take(c, keep ? 4 * N : 0);
  L.off_dchi64 = take(c, keep ? 8 * N : 0);
  L.off_lam64 = take(c, keep ? 16 * N : 0);
  L.off_lam32 = take(c, keep ? 4 * N : 0);
  const size_t half = (size_t)(R / 2 + 1);
  // x, b per coarse level (and a Jacobi buffer t for the unlumped operator)
  const size_t lev = (opt.galerkin ? 3 : 2) * (half * half * half * 8 / 7 + 64 * kMaxLevels + 64);
  L.off_levels = take(c, 4 * lev);
  L.off_dct = take(c, 8 * (512 + 160 + 512 + 16 + 512 + 520) + 4 * (512 + 512));   // spectral tables, n <= 512
  const size_t Pp = (size_t)(P > 0 ? P : 1);
  L.off_pcell = take(c, 4 * Pp);
  L.off_pfrac = take(c, 16 * Pp);
  L.off_pnrm = take(c, keep ? 16 * Pp : 0);
  L.off_srec = take(c, 32 * Pp);
  const size_t nt = (size_t)div_up(R, kSplatTile);
  const size_t ntiles = nt * nt * nt;
  L.off_tile_count = take(c, 4 * (ntiles + 1));
  L.off_tile_off = take(c, 4 * (ntiles + 2));
  L.off_tile_cursor = take(c, 4 * (ntiles + 1));
  const int nb = div_up(R - 1, kBrick);
  const size_t nbricks = (size_t)nb * nb * nb;
  L.off_brick_count = take(c, 4 * (nbricks + 1));
  L.off_brick_off = take(c, 4 * (nbricks + 2));
  L.off_leaf_off = take(c, 4 * (8 * nbricks + 2));
  L.off_leaf_cnt = take(c, 4 * 8 * nbricks);
  int64_t cap = opt.mesh_capacity > 0 ? opt.mesh_capacity : (int64_t)16 * R * R;
  if (cap < 4096) cap = 4096;
  L.cap = cap;
  L.off_tris = take(c, sizeof(Tri) * (size_t)cap);
  L.off_tris_lo = take(c, keep ? sizeof(Tri) * (size_t)cap : 0);
  L.off_tris_s = take(c, sizeof(float4) * kTriRec * (size_t)cap);
  L.off_cell_pyr = take(c, 2 * sizeof(float4) * (size_t)cap);
  L.off_pyr = take(c, 32 * pyramid_nodes(nb));
  L.off_pyr_sums = take(c, 32 * pyramid_aux_nodes(nb));
  L.off_pyr_rth = take(c, 8 * pyramid_aux_nodes(nb));
  // per-block partial pairs: splat tiles, the refinement pass (one block per
  // 64 x 8 cells of a plane), fixed-size reductions, SH adjoint
  const size_t resid_blocks = (size_t)div_up(R, 64) * div_up(R, 8) * R;
  L.n_partials = std::max<size_t>(std::max<size_t>(2 * ntiles, 2 * resid_blocks),
                                  std::max<size_t>(4 * kPartials, 81 * 256));
  L.off_partials = take(c, 8 * L.n_partials);
  L.n_scan = scan_tmp_size((int)std::max(ntiles, nbricks));
  L.off_scan = take(c, 4 * L.n_scan);
  L.off_state = take(c, sizeof(DevState));
  // normal estimation: per point a cell, a key and two float4 copies, per
  // kDpcaBox points a box, per cell a count, an offset and a cursor
  // the same buffers sort exact queries, in chunks of Pd: up to 2^20 (one
  // chunk for a million queries on large grids, where a chunk of a few
  // hundred thousand leaves the search with too few warps per wave)
  const size_t Pd = std::max<size_t>(Pp, std::min<size_t>((size_t)1 << 20, std::max<size_t>(65536, N / 4)));
  L.dp_points = (int64_t)Pd;
  L.dp_cap = point_grid_cap((int64_t)Pd);
  L.off_dp_cell = take(c, 4 * Pd);
  L.off_dp_tmp = take(c, 16 * Pd);
  L.off_dp_sorted = take(c, 16 * Pd);
  L.off_dp_count = take(c, 4 * ((size_t)L.dp_cap + 1));
  L.off_dp_off = take(c, 4 * ((size_t)L.dp_cap + 2));
  L.off_dp_cursor = take(c, 4 * ((size_t)L.dp_cap + 1));
  L.off_dp_key = take(c, 4 * Pd);
  L.off_dp_gbox = take(c, 32 * ((Pd + kDpcaBox - 1) / kDpcaBox));
  L.off_or_scal = take(c, 16 * sizeof(unsigned));
  L.n_dp_scan = scan_tmp_size((int)L.dp_cap);
  L.off_dp_scan = take(c, 4 * L.n_dp_scan);
  L.total = (c + kAlign - 1) / kAlign * kAlign;
  return L;
}

bool valid_opt(const wgeo_options& o) {
  return o.tol_rel >= 0.0 && o.tol_rel_adjoint >= 0.0 && o.max_vcycles >= 0 && o.max_vcycles <= 1000 &&
         o.max_refine >= 0 &&
         o.max_refine <= 200 && o.vcycles_per_refine >= 1 && o.vcycles_per_refine <= 20 &&
         (o.precision == WGEO_PREC_MIXED || o.precision == WGEO_PREC_FP32 || o.precision == WGEO_PREC_FP64) &&
         o.mesh_capacity >= 0 &&
         (o.galerkin == 0 || (o.galerkin == 1 && o.precision == WGEO_PREC_MIXED)) &&
         (o.spectral == 0 || o.spectral == 1) &&
         o.mesh_capacity < (int64_t)1 << 31;
}

__global__ void reset_status_kernel(DevState* st) {
  st->status = 0;
  st->ntris = 0;
  st->c = 0.0;
  st->c_up = 0.f;
  st->npts = 0;
  st->sdf_cnt[0] = 0;
  st->sdf_cnt[1] = 0;
  st->sdf_cnt[2] = 0;
  st->sdf_cnt[3] = 0;
  st->nmax_bits = 0;
}

void accumulate_slot(StageTimer& t, int slot) {
  if (!t.used[slot]) return;
  cudaEventSynchronize(t.end[slot]);
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, t.beg[slot], t.end[slot]) == cudaSuccess) {
    t.acc_ms += ms;
    t.count += 1;
  }
  t.used[slot] = false;
}

}  // namespace

namespace wgeo {

std::atomic<long long> g_kernel_launches{0};
thread_local long long t_kernel_launches = 0;

int stage_begin(wgeo_handle* h, int stage, cudaStream_t s) {
  if (!h->opt.stage_timing) return -1;
  if (!h->timers) {
    h->timers = new (std::nothrow) StageTimer[kStages]();
    if (!h->timers) return -1;
  }
  StageTimer& t = h->timers[stage];
  const int slot = t.head;
  t.head = (t.head + 1) % kRing;
  accumulate_slot(t, slot);   // ring full: fold the oldest pair in first
  if (!t.beg[slot]) {
    if (cudaEventCreate(&t.beg[slot]) != cudaSuccess) return -1;
    if (cudaEventCreate(&t.end[slot]) != cudaSuccess) return -1;
  }
  if (cudaEventRecord(t.beg[slot], s) != cudaSuccess) return -1;
  return slot;
}

void stage_end(wgeo_handle* h, int stage, int slot, cudaStream_t s) {
  if (slot < 0 || !h->timers) return;
  StageTimer& t = h->timers[stage];
  if (cudaEventRecord(t.end[slot], s) == cudaSuccess) t.used[slot] = true;
}

}  // namespace wgeo

extern "C" {

int64_t wgeo_kernel_launches(void) {
  return (int64_t)g_kernel_launches.load(std::memory_order_relaxed) + (int64_t)loop_launches();
}

int wgeo_stage_times(wgeo_handle* h, double* ms, int64_t* counts, int32_t reset) {
  if (!h || !ms || !counts) return WGEO_ERR_INVALID_ARG;
  if (!h->timers) return WGEO_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  for (int s = 0; s < kStages; ++s) {
    StageTimer& t = h->timers[s];
    for (int k = 0; k < kRing; ++k) accumulate_slot(t, k);
    ms[s] += t.acc_ms;
    counts[s] += t.count;
    if (reset) {
      t.acc_ms = 0.0;
      t.count = 0;
    }
  }
  return WGEO_OK;
}

int wgeo_default_options(wgeo_options* opt) {
  if (!opt) return WGEO_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->tol_rel = 1e-6;
  opt->max_vcycles = 40;
  opt->max_refine = 10;
  opt->vcycles_per_refine = 2;
  opt->precision = WGEO_PREC_MIXED;
  opt->warm_start = 0;
  opt->keep_for_backward = 1;
  opt->mesh_capacity = 0;
  opt->use_graphs = 1;
  opt->spectral = 1;
  opt->tol_rel_adjoint = 1e-7;
  return WGEO_OK;
}

size_t wgeo_footprint_bytes(int32_t max_res, int64_t max_points, const wgeo_options* opt) {
  wgeo_options o;
  if (opt) o = *opt; else wgeo_default_options(&o);
  if (!valid_res(max_res) || max_points < 0 || !valid_opt(o)) return 0;
  return make_layout(max_res, max_points, o).total;
}

int wgeo_create(wgeo_handle** out, int32_t max_res, int64_t max_points, const wgeo_options* opt) {
  if (!out) return WGEO_ERR_INVALID_ARG;
  *out = nullptr;
  wgeo_options o;
  if (opt) o = *opt; else wgeo_default_options(&o);
  if (!valid_res(max_res) || max_points < 0 || max_points > ((int64_t)1 << 30) || !valid_opt(o))
    return WGEO_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WGEO_ERR_NOT_BUILT_FOR_DEVICE;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major * 10 + minor != 103) return WGEO_ERR_NOT_BUILT_FOR_DEVICE;
  const Layout L = make_layout(max_res, max_points, o);
  wgeo_handle* h = new (std::nothrow) wgeo_handle();
  if (!h) return WGEO_ERR_OOM;
  h->max_res = max_res;
  h->max_points = max_points;
  h->opt = o;
  h->device = dev;
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || h->num_sms < 1) {
    cudaGetLastError();
    delete h;
    return WGEO_ERR_CUDA;
  }
  if (cudaMalloc(&h->arena, L.total) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return WGEO_ERR_OOM;
  }
  h->arena_bytes = L.total;
  char* a = h->arena;
  const bool keep = o.keep_for_backward != 0;
  const size_t N = (size_t)max_res * max_res * max_res;
  h->b32 = (float*)(a + L.off_b32);
  h->chi32 = (float*)(a + L.off_chi32);
  h->chiff[0] = (float2*)(a + L.off_chi64);
  h->chiff[1] = h->chiff[0] + N;
  h->r32 = (float*)(a + L.off_r32);
  h->e32 = (float*)(a + L.off_e32);
  h->phi = (float*)(a + L.off_phi);
  h->ctri = keep ? (int*)(a + L.off_ctri) : nullptr;
  h->dphi = keep ? (float*)(a + L.off_dphi) : nullptr;
  h->dchi64 = keep ? (double*)(a + L.off_dchi64) : nullptr;
  h->lamff[0] = keep ? (float2*)(a + L.off_lam64) : nullptr;
  h->lamff[1] = keep ? h->lamff[0] + N : nullptr;
  h->lam32 = keep ? (float*)(a + L.off_lam32) : nullptr;
  h->level_pool = (float*)(a + L.off_levels);
  h->dct_t1 = (float2*)(a + L.off_dct);
  h->dct_w32 = h->dct_t1 + 512;
  h->dct_wml = h->dct_w32 + 160;
  h->dct_tr = h->dct_wml + 512;
  h->dct_sk = (float*)(h->dct_tr + 16);
  h->dct_skl = h->dct_sk + 512;
  h->dct_tw = reinterpret_cast<float2*>(h->dct_skl + 512);
  h->dct_wq = h->dct_tw + 512;
  h->pcell = (int*)(a + L.off_pcell);
  h->pfrac = (float4*)(a + L.off_pfrac);
  h->pnrm = keep ? (float4*)(a + L.off_pnrm) : nullptr;
  h->srec = (float4*)(a + L.off_srec);
  h->tile_count = (int*)(a + L.off_tile_count);
  h->tile_off = (int*)(a + L.off_tile_off);
  h->tile_cursor = (int*)(a + L.off_tile_cursor);
  h->brick_count = (int*)(a + L.off_brick_count);
  h->brick_off = (int*)(a + L.off_brick_off);
  h->leaf_off = (int*)(a + L.off_leaf_off);
  h->leaf_cnt = (unsigned*)(a + L.off_leaf_cnt);
  h->mesh_cap = L.cap;
  h->tris = (Tri*)(a + L.off_tris);
  h->tris_lo = keep ? (Tri*)(a + L.off_tris_lo) : nullptr;
  h->tris_s = (float4*)(a + L.off_tris_s);
  h->cell_pyr = (float4*)(a + L.off_cell_pyr);
  h->pyramid = (float4*)(a + L.off_pyr);
  h->pyr_sums = (float4*)(a + L.off_pyr_sums);
  h->pyr_rth = (unsigned*)(a + L.off_pyr_rth);
  h->partials = (double*)(a + L.off_partials);
  h->scan_tmp = (int*)(a + L.off_scan);
  h->scan_tmp_elems = L.n_scan;
  h->dstate = (DevState*)(a + L.off_state);
  h->dp_cell_cap = L.dp_cap;
  h->dp_points = L.dp_points;
  h->dp_cell = (int*)(a + L.off_dp_cell);
  h->dp_tmp = (float4*)(a + L.off_dp_tmp);
  h->dp_sorted = (float4*)(a + L.off_dp_sorted);
  h->dp_count = (int*)(a + L.off_dp_count);
  h->dp_off = (int*)(a + L.off_dp_off);
  h->dp_cursor = (int*)(a + L.off_dp_cursor);
  h->dp_key = (int*)(a + L.off_dp_key);
  h->dp_gbox = (float4*)(a + L.off_dp_gbox);
  h->or_scal = (unsigned*)(a + L.off_or_scal);
  h->dp_scan = (int*)(a + L.off_dp_scan);
  if (upload_mc_table() != WGEO_OK || cudaMemset(h->dstate, 0, sizeof(DevState)) != cudaSuccess ||
      cudaMemset(h->chiff[0], 0, 16 * N) != cudaSuccess) {
    cudaFree(h->arena);
    delete h;
    return WGEO_ERR_CUDA;
  }
  *out = h;
  return WGEO_OK;
}

int wgeo_destroy(wgeo_handle* h) {
  if (!h) return WGEO_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->timers) {
    for (int s = 0; s < kStages; ++s)
      for (int k = 0; k < kRing; ++k) {
        if (h->timers[s].beg[k]) cudaEventDestroy(h->timers[s].beg[k]);
        if (h->timers[s].end[k]) cudaEventDestroy(h->timers[s].end[k]);
      }
    delete[] h->timers;
  }
  cudaFree(h->arena);
  delete h;
  return WGEO_OK;
}

int wgeo_reconstruct(wgeo_handle* h, const float* points, const float* normals, int64_t n,
                     const float* bbox, int32_t res, float* sdf_out, float* nrm_out, void* stream) {
  if (!h || !bbox || n < 0 || n > h->max_points) return WGEO_ERR_INVALID_ARG;
  if (n > 0 && (!points || !normals)) return WGEO_ERR_INVALID_ARG;
  if (!valid_res(res) || res > h->max_res) return WGEO_ERR_INVALID_ARG;
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (!isfinite(bbox[a]) || !isfinite(bbox[a + 3]) || !(bbox[a + 3] > bbox[a])) return WGEO_ERR_INVALID_ARG;
    ext = fmax(ext, (double)bbox[a + 3] - (double)bbox[a]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  const bool same_res = (h->res == res);
  if (!same_res || h->nlevels == 0) {
    int rc = build_levels(h, res);
    if (rc) return rc;
  }
  h->res = res;
  h->h = ext / res;
  for (int a = 0; a < 3; ++a) h->lo[a] = (double)bbox[a];
  h->npts = n;
  h->have_forward = false;
  const int64_t N = (int64_t)res * res * res;
  reset_status_kernel<<<1, 1, 0, s>>>(h->dstate);
  WGEO_LAUNCH_CHECK();
  const bool warm = h->opt.warm_start && h->chi_valid_for_warm && h->warm_res == res;
  if (!warm && h->opt.precision == WGEO_PREC_FP32) WGEO_CUDA_TRY(cudaMemsetAsync(h->chi32, 0, 4 * N, s));
  int slot = stage_begin(h, kStSplat, s);
  int rc = launch_bin_sort_splat(h, points, normals, n, res, s);
  if (rc) return rc;
  stage_end(h, kStSplat, slot, s);
  slot = stage_begin(h, kStSolve, s);
  rc = launch_solve(h, res, 0, !warm, s);
  if (rc) return rc;
  stage_end(h, kStSolve, slot, s);
  slot = stage_begin(h, kStIso, s);
  rc = launch_isovalue(h, points, n, res, s);
  if (rc) return rc;
  stage_end(h, kStIso, slot, s);
  rc = launch_mc_sdf_normals(h, res, sdf_out, nrm_out, s);
  if (rc) return rc;
  h->chi_valid_for_warm = true;
  h->warm_res = res;
  h->have_forward = true;
  h->last_stream = s;
  return WGEO_OK;
}

int wgeo_query(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* nrm_q, void* stream) {
  if (!h || m < 0) return WGEO_ERR_INVALID_ARG;
  if (m > 0 && (!q || !sdf_q)) return WGEO_ERR_INVALID_ARG;
  if (!h->have_forward) return WGEO_ERR_NO_FORWARD;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = stage_begin(h, kStQuery, s);
  int rc = launch_query(h, q, m, sdf_q, nrm_q, s);
  stage_end(h, kStQuery, slot, s);
  h->last_stream = s;
  return rc;
}

int wgeo_query_exact(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* grad_q, void* stream) {
  if (!h || m < 0) return WGEO_ERR_INVALID_ARG;
  if (m > 0 && (!q || !sdf_q)) return WGEO_ERR_INVALID_ARG;
  if (!h->have_forward) return WGEO_ERR_NO_FORWARD;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = stage_begin(h, kStQueryExact, s);
  int rc = launch_query_exact(h, q, m, sdf_q, grad_q, s);
  stage_end(h, kStQueryExact, slot, s);
  h->last_stream = s;
  return rc;
}

int wgeo_backward(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                  const float* d_sdf_q, const float* d_nrm_q, int64_t m, float* d_points,
                  float* d_normals, float* d_q, void* stream) {
  if (!h || m < 0) return WGEO_ERR_INVALID_ARG;
  if (!h->have_forward || !h->opt.keep_for_backward) return WGEO_ERR_NO_FORWARD;
  if (h->npts > 0 && (!d_points || !d_normals)) return WGEO_ERR_INVALID_ARG;
  if (m > 0 && (d_sdf_q || d_nrm_q || d_q) && !q) return WGEO_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = launch_backward(h, d_sdf_grid, d_nrm_grid, q, d_sdf_q, d_nrm_q, m, d_points, d_normals, d_q, s);
  h->last_stream = s;
  return rc;
}

int wgeo_estimate_normals(wgeo_handle* h, const float* points, int64_t n, const float* bbox, float radius,
                          float eps, float* normals, int32_t* counts, void* stream) {
  if (!h || !bbox || n < 0 || n > h->max_points) return WGEO_ERR_INVALID_ARG;
  if (n > 0 && (!points || !normals)) return WGEO_ERR_INVALID_ARG;
  if (!(isfinite(radius) && radius > 0.f && isfinite(eps) && eps >= 1e-6f * radius)) return WGEO_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(bbox[a]) || !isfinite(bbox[a + 3]) || !(bbox[a + 3] >= bbox[a])) return WGEO_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = stage_begin(h, kStPointPca, s);
  int rc = launch_dpca(h, points, n, bbox, radius, eps, normals, counts, s);
  stage_end(h, kStPointPca, slot, s);
  h->last_stream = s;
  return rc;
}

int wgeo_orient_normals(wgeo_handle* h, const float* points, int64_t n, const float* bbox, float gamma,
                        int32_t n_tol, float* normals, int32_t* stats, float* rd_out, void* stream) {
  if (!h || !bbox || n < 0 || n > h->max_points) return WGEO_ERR_INVALID_ARG;
  if (n > 0 && (!points || !normals)) return WGEO_ERR_INVALID_ARG;
  if (!(isfinite(gamma) && gamma >= 1.f) || n_tol < 0) return WGEO_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(bbox[a]) || !isfinite(bbox[a + 3]) || !(bbox[a + 3] >= bbox[a])) return WGEO_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = stage_begin(h, kStOrient, s);
  int rc = launch_orient(h, points, n, bbox, gamma, n_tol, normals, stats, rd_out, s);
  stage_end(h, kStOrient, slot, s);
  h->last_stream = s;
  return rc;
}

int wgeo_backward_exact(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                        const float* d_sdf_q, int64_t m, float* d_points, float* d_normals, float* d_q,
                        void* stream) {
  if (!h || m < 0) return WGEO_ERR_INVALID_ARG;
  if (!h->have_forward || !h->opt.keep_for_backward) return WGEO_ERR_NO_FORWARD;
  if (h->npts > 0 && (!d_points || !d_normals)) return WGEO_ERR_INVALID_ARG;
  if (m > 0 && (d_sdf_q || d_q) && !q) return WGEO_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = launch_backward_exact(h, d_sdf_grid, d_nrm_grid, q, d_sdf_q, m, d_points, d_normals, d_q, s);
  h->last_stream = s;
  return rc;
}

int wgeo_get_info(wgeo_handle* h, wgeo_info* out) {
  if (!h || !out) return WGEO_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return WGEO_ERR_CUDA;
  DevState st;
  if (cudaMemcpy(&st, h->dstate, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return WGEO_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  out->status = st.status;
  out->res = h->res;
  out->solver_steps = st.fwd.iter;
  out->backward_steps = st.bwd.iter;
  out->residual_rel = st.fwd.rel;
  out->backward_residual_rel = st.bwd.rel;
  out->isovalue = st.c;
  out->n_triangles = st.ntris;
  out->n_points_used = st.npts;
  out->h = h->h;
  out->sdf_node_visits = (int64_t)st.sdf_cnt[0];
  out->sdf_leaf_visits = (int64_t)st.sdf_cnt[1];
  out->sdf_tri_tests = (int64_t)st.sdf_cnt[2];
  out->sdf_tie_nodes = (int64_t)st.sdf_cnt[3];
  out->backward_dc = st.dc;
  return WGEO_OK;
}

int64_t wgeo_get_field(wgeo_handle* h, int32_t which, float* out, void* stream) {
  if (!h || !out) return -WGEO_ERR_INVALID_ARG;
  if (!h->have_forward) return -WGEO_ERR_NO_FORWARD;
  const int64_t N = (int64_t)h->res * h->res * h->res;
  if (cudaSetDevice(h->device) != cudaSuccess) return -WGEO_ERR_CUDA;
  if (which >= 3 && which <= 5) {
    if (!h->opt.keep_for_backward) return -WGEO_ERR_NO_FORWARD;
    const int rc = launch_export_adjoint(h, which, out, (cudaStream_t)stream);
    return rc ? -rc : N;
  }
  if (which == 6 && !h->opt.keep_for_backward) return -WGEO_ERR_NO_FORWARD;
  const void* src = which == 0 ? (const void*)h->b32 : which == 1 ? (const void*)h->chi32
                  : which == 2 ? (const void*)h->phi : which == 6 ? (const void*)h->ctri : nullptr;
  if (!src) return -WGEO_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(out, src, 4 * N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
    return -WGEO_ERR_CUDA;
  return N;
}

int64_t wgeo_get_bins(wgeo_handle* h, int32_t* cells, void* stream) {
  if (!h || !cells) return -WGEO_ERR_INVALID_ARG;
  if (!h->have_forward) return -WGEO_ERR_NO_FORWARD;
  if (cudaSetDevice(h->device) != cudaSuccess) return -WGEO_ERR_CUDA;
  const int rc = launch_unpack_bins(h, cells, (cudaStream_t)stream);
  if (rc) return -rc;
  return h->npts;
}

int64_t wgeo_get_mesh(wgeo_handle* h, float* verts, int64_t* edge_ids, int64_t cap) {
  if (!h || cap < 0) return -WGEO_ERR_INVALID_ARG;
  if (!h->have_forward) return -WGEO_ERR_NO_FORWARD;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return -WGEO_ERR_CUDA;
  DevState st;
  if (cudaMemcpy(&st, h->dstate, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return -WGEO_ERR_CUDA;
  const int64_t T = st.ntris;
  int64_t k = T < cap ? T : cap;
  if (k > h->mesh_cap) k = h->mesh_cap;
  if (k > 0 && (verts || edge_ids)) {
    Tri* tmp = new (std::nothrow) Tri[k];
    if (!tmp) return -WGEO_ERR_OOM;
    if (cudaMemcpy(tmp, h->tris, sizeof(Tri) * k, cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete[] tmp;
      return -WGEO_ERR_CUDA;
    }
    for (int64_t t = 0; t < k; ++t) {
      const float4 v[3] = {tmp[t].a, tmp[t].b, tmp[t].c};
      for (int q = 0; q < 3; ++q) {
        if (verts) {
          verts[(t * 3 + q) * 3 + 0] = v[q].x;
          verts[(t * 3 + q) * 3 + 1] = v[q].y;
          verts[(t * 3 + q) * 3 + 2] = v[q].z;
        }
        if (edge_ids) {
          int gid;
          memcpy(&gid, &v[q].w, sizeof(int));
          edge_ids[t * 3 + q] = gid;
        }
      }
    }
    delete[] tmp;
  }
  return T;
}

int wgeo_mc_table(int32_t* counts, int32_t* tris) {
  if (!counts || !tris) return WGEO_ERR_INVALID_ARG;
  host_mc_table(counts, tris);
  return WGEO_OK;
}

int wgeo_sh_surface(const float* theta, int32_t K, const float* dirs, int64_t n, float base,
                    const float* centre, float* points, float* normals, void* stream) {
  if (!sh_valid_K(K) || n < 0 || !theta || !centre || (n > 0 && (!dirs || !points || !normals)))
    return WGEO_ERR_INVALID_ARG;
  return launch_sh_surface(theta, K, dirs, n, base, centre, points, normals, (cudaStream_t)stream);
}

int wgeo_sh_surface_backward(wgeo_handle* h, const float* theta, int32_t K, const float* dirs, int64_t n,
                             float base, const float* d_points, const float* d_normals, float* d_theta,
                             void* stream) {
  if (!h || !sh_valid_K(K) || n < 0 || !theta || !d_theta ||
      (n > 0 && (!dirs || !d_points || !d_normals)))
    return WGEO_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return WGEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = launch_sh_backward(h, theta, K, dirs, n, base, d_points, d_normals, d_theta, s);
  h->last_stream = s;
  return rc;
}

const char* wgeo_error_string(int code) {
  switch (code) {
    case WGEO_OK: return "ok";
    case WGEO_ERR_INVALID_ARG: return "invalid argument";
    case WGEO_ERR_OOM: return "device out of memory";
    case WGEO_ERR_CUDA: return "CUDA error";
    case WGEO_ERR_NO_FORWARD: return "no forward state on this handle";
    case WGEO_ERR_NOT_BUILT_FOR_DEVICE: return "no sm_103a device";
    default: return "unknown error";
  }
}

const char* wgeo_status_string(uint32_t bits) {
  if (bits == 0) return "ok";
  if (bits & WGEO_STATUS_MESH_CAPACITY) return "mesh capacity exceeded";
  if (bits & WGEO_STATUS_NONFINITE_INPUT) return "non-finite input point or normal";
  if (bits & WGEO_STATUS_EMPTY_SURFACE) return "empty surface";
  if (bits & WGEO_STATUS_NOT_CONVERGED) return "solver not converged";
  if (bits & WGEO_STATUS_POINT_OUTSIDE_BBOX) return "point outside bounding box";
  return "unknown status";
}

}  // extern "C"
