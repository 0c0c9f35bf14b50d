// Distance-weighted PCA normal estimation (Sec. 2.1): for every point x_i,
// the neighbourhood N_i = { x_j : |x_j - x_i| <= R } (x_i included), weights
// w_ij = 1 / (|x_j - x_i| + eps), the weighted centroid, the weighted
// covariance C_i (Eq. weighted_covariance) and n_i = the eigenvector of C_i
// with the smallest eigenvalue (unit, unoriented).  Fewer than 3 neighbours,
// or a covariance without a positive eigenvalue, gives the zero vector.
//
// Layout.  Points are binned into cubic cells of edge >= R over the box
// (points outside it are clamped into the edge cells: clamping never moves
// two points' cells further apart than their distance allows, so the 27 cells
// around a point's cell still hold its whole neighbourhood).  A counting sort
// groups them by cell, and a rank pass puts each cell's entries in point-
// index order, so every sum below runs in one fixed order and the result does
// not depend on the order in which atomics landed.  One thread per point, in
// sorted order, so that the lanes of a warp mostly share their 27 cells.
//
// Arithmetic.  Membership is decided in float32 with every operation rounded
// ((dx^2 + dy^2) + dz^2 against R^2, no contraction into FMA), the precision
// in which the paper's kernels decide it.  The moments are taken relative to
// x_i and scaled by 1/R: with y = (x_j - x_i) / R, S0 = sum w, m = sum w y / S0
// and S2 = sum w y y^T, C = S2 / S0 - m m^T is C_i / R^2 (the centred
// covariance written by the moment identity; same eigenvectors).  The 3 x 3
// symmetric eigenproblem is solved by cyclic Jacobi rotations (Golub and Van
// Loan, Matrix Computations, the symmetric Schur decomposition of each
// off-diagonal pair in turn).
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

// Cell of every point and the per-cell counts; points with a non-finite
// coordinate join no cell (and get the zero normal here when normals is set).
__global__ void dpca_bin_kernel(const float* __restrict__ pts, int n, PointGrid g, int* __restrict__ cell_of,
                                int* __restrict__ count, float* __restrict__ normals) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float x = pts[3 * (int64_t)i], y = pts[3 * (int64_t)i + 1], z = pts[3 * (int64_t)i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
      cell_of[i] = -1;
      if (normals) {
        normals[3 * (int64_t)i] = 0.f;
        normals[3 * (int64_t)i + 1] = 0.f;
        normals[3 * (int64_t)i + 2] = 0.f;
      }
      continue;
    }
    const int cell = grid_cell(g, x, y, z);
    cell_of[i] = cell;
    atomicAdd(&count[cell], 1);
  }
}

// Position of a point inside its cell as a 9-bit Morton key of an 8 x 8 x 8
// split of the cell (coordinates outside the cell clamp to its faces).
__device__ __forceinline__ int dpca_subkey(const PointGrid& g, float x, float y, float z) {
  const float p[3] = {x, y, z};
  int c[3];
  grid_cell3(g, x, y, z, c);
  int key = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float t = ((p[a] - g.lo[a]) * g.inv_cs - (float)c[a]) * 8.f;
    const int s = (int)fminf(fmaxf(floorf(t), 0.f), 7.f);
    key |= ((s & 1) | ((s & 2) << 2) | ((s & 4) << 4)) << a;
  }
  return key;
}

// Unordered scatter into the cells' ranges: (x, y, z, point index bits) and
// the entry's sub-cell key.
__global__ void dpca_scatter_kernel(const float* __restrict__ pts, int n, PointGrid g,
                                    const int* __restrict__ cell_of, const int* __restrict__ off,
                                    int* __restrict__ cursor, float4* __restrict__ tmp, int* __restrict__ tkey) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int cell = cell_of[i];
    if (cell < 0) continue;
    const int pos = off[cell] + atomicAdd(&cursor[cell], 1);
    const float x = pts[3 * (int64_t)i], y = pts[3 * (int64_t)i + 1], z = pts[3 * (int64_t)i + 2];
    tmp[pos] = make_float4(x, y, z, __int_as_float(i));
    tkey[pos] = dpca_subkey(g, x, y, z);
  }
}

// Each entry moves to its rank by (sub-cell key, point index) within its
// cell's range: a fixed order in which consecutive entries lie close together.
__global__ void dpca_rank_kernel(const float4* __restrict__ tmp, const int* __restrict__ tkey,
                                 const int* __restrict__ cell_of, const int* __restrict__ off,
                                 const int* __restrict__ total, float4* __restrict__ sorted) {
  const int m = *total;
  const int* tidx = reinterpret_cast<const int*>(tmp) + 3;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m; p += gridDim.x * blockDim.x) {
    const float4 v = tmp[p];
    const int idx = __float_as_int(v.w), key = tkey[p];
    const int cell = cell_of[idx];
    const int s0 = off[cell], s1 = off[cell + 1];
    int rank = 0;
    for (int j = s0; j < s1; ++j) {
      const int kj = tkey[j];
      rank += kj < key || (kj == key && tidx[4 * (int64_t)j] < idx);
    }
    sorted[s0 + rank] = v;
  }
}

// Bounding box of each group of kDpcaBox consecutive sorted entries (the last
// group may be partial): box[2 g] = min corner, box[2 g + 1] = max corner.
// One half-warp per group.
__global__ void dpca_group_box_kernel(const float4* __restrict__ sorted, const int* __restrict__ total,
                                      float4* __restrict__ box) {
  static_assert(kDpcaBox == 16, "one half-warp per group");
  const int m = *total;
  const int sub = threadIdx.x & 15;
  const int nhalf = gridDim.x * (blockDim.x >> 4);
  // every lane of a warp runs the same number of iterations (shuffles below)
  const int first = blockIdx.x * (blockDim.x >> 4) + ((threadIdx.x >> 5) << 1);
  for (int pair = first; pair * kDpcaBox < m; pair += nhalf) {
    const int grp = pair + ((threadIdx.x >> 4) & 1);
    const int k = grp * kDpcaBox + sub;
    const float4 v = sorted[k < m ? k : pair * kDpcaBox];
    float lo[3] = {v.x, v.y, v.z}, hi[3] = {v.x, v.y, v.z};
    if (grp * kDpcaBox >= m) {   // the second half of the last pair: nothing to bound
      lo[0] = lo[1] = lo[2] = INFINITY;
      hi[0] = hi[1] = hi[2] = -INFINITY;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
        hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
      }
    if (sub == 0 && grp * kDpcaBox < m) {
      box[2 * grp] = make_float4(lo[0], lo[1], lo[2], 0.f);
      box[2 * grp + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
  }
}

// Unit eigenvector of the smallest eigenvalue of the symmetric 3 x 3 matrix a
// (overwritten), and the largest eigenvalue.
__device__ __forceinline__ float jacobi_min_vector(float a[3][3], float v_out[3]) {
  float v[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  const float scale = fabsf(a[0][0]) + fabsf(a[1][1]) + fabsf(a[2][2]) + fabsf(a[0][1]) + fabsf(a[0][2]) +
                      fabsf(a[1][2]);
#pragma unroll 1
  for (int sweep = 0; sweep < 10; ++sweep) {
    const float off = fabsf(a[0][1]) + fabsf(a[0][2]) + fabsf(a[1][2]);
    if (!(off > 1e-9f * scale)) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;   // pairs (0,1), (0,2), (1,2)
      const float apq = a[p][q];
      if (!(fabsf(apq) > 1e-12f * scale)) {
        a[p][q] = a[q][p] = 0.f;
        continue;
      }
      // tan of the angle that zeroes a_pq: the smaller root of
      // t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 a_pq)
      const float tau = (a[q][q] - a[p][p]) / (2.f * apq);
      const float t = fabsf(tau) < 1e18f ? copysignf(1.f, tau) / (fabsf(tau) + sqrtf(tau * tau + 1.f))
                                         : 0.5f / tau;
      const float c = rsqrtf(t * t + 1.f), s = t * c;
      // a <- J^T a J with J the rotation (J_pp = J_qq = c, J_pq = s, J_qp = -s)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
      a[p][q] = a[q][p] = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
  // column of the smallest diagonal entry (selects, not a runtime index, keep
  // everything in registers)
  float e = a[0][0], x = v[0][0], y = v[1][0], z = v[2][0];
  if (a[1][1] < e) {
    e = a[1][1];
    x = v[0][1];
    y = v[1][1];
    z = v[2][1];
  }
  if (a[2][2] < e) {
    x = v[0][2];
    y = v[1][2];
    z = v[2][2];
  }
  const float nrm = rsqrtf(x * x + y * y + z * z);
  v_out[0] = x * nrm;
  v_out[1] = y * nrm;
  v_out[2] = z * nrm;
  return fmaxf(a[0][0], fmaxf(a[1][1], a[2][2]));
}

// Work split.  A warp takes a chunk of kDpcaPts = 8 consecutive sorted points
// (they lie close together) from a counter, so dense regions leave no tail of
// idle SMs; each point has kDpcaLanes = 4 lanes, and lane s of a point handles
// the entries whose sorted index is s mod 4.  The four partial sums are then
// added in a fixed butterfly order, identical on the four lanes.
//
// Candidates.  Each lane works out which cells its point's ball can reach: in
// cell units, with its coordinate u clamped into [0, dim] (clamping only
// shortens distances, as it does for the cells of points outside the box),
// the rows (cy, cz) whose slab lies within rc of u and, in each, the x cells
// within the rest of rc.  The warp visits the union of these ranges row by
// row, in the groups of kDpcaBox entries that overlap them; a group runs only
// when some point's ball reaches the group's bounding box.  The box test
// repeats the membership test's float operations on the box's clamped
// differences, and rounding is monotone, so it never drops a group holding an
// accepted entry.  A rejected entry adds exact zeros, and a lane's accepted
// entries come in the same order whatever else its warp holds, so the result
// of a point does not depend on the warp's make-up.  rc = R / cell edge plus
// a margin for the rounding of cell coordinates and of the membership test.
//
// Weights.  w' = R w = 1 / (d / R + eps / R), at most R / eps <= 1e6, from the
// hardware square root and reciprocal (relative error ~1e-7; weights decide
// nothing, they only scale the moments).
__device__ __forceinline__ float approx_sqrt(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float approx_rcp(float x) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(128, 4) dpca_normal_kernel(const float4* __restrict__ sorted,
                                                          const int* __restrict__ off,
                                                          const int* __restrict__ total, PointGrid g,
                                                          const float4* __restrict__ gbox, int* __restrict__ next,
                                                          float radius, float eps_r, float rc,
                                                          float* __restrict__ normals, int* __restrict__ counts) {
  constexpr unsigned kFull = 0xffffffffu;
  const int m = *total;
  const int lane = threadIdx.x & 31;
  const int sl = lane & (kDpcaLanes - 1);   // sub-lane of the point
  const float r2 = __fmul_rn(radius, radius), inv_r = 1.f / radius;
  const float rc2 = rc * rc;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(next, 1);
    const int base = __shfl_sync(kFull, chunk, 0) * kDpcaPts;
    if (base >= m) break;
    const int k = base + lane / kDpcaLanes;
    const bool valid = k < m;
    const float4 q = sorted[valid ? k : base];   // spare points mirror the chunk's first
    float u[3];
    {
      const float p[3] = {q.x, q.y, q.z};
#pragma unroll
      for (int a = 0; a < 3; ++a) u[a] = fminf(fmaxf((p[a] - g.lo[a]) * g.inv_cs, 0.f), (float)g.dim[a]);
    }
    const int z0 = __reduce_min_sync(kFull, max((int)floorf(u[2] - rc), 0));
    const int z1 = __reduce_max_sync(kFull, min((int)floorf(u[2] + rc), g.dim[2] - 1));
    const int y0 = __reduce_min_sync(kFull, max((int)floorf(u[1] - rc), 0));
    const int y1 = __reduce_max_sync(kFull, min((int)floorf(u[1] + rc), g.dim[1] - 1));
    float S0 = 0.f, S1x = 0.f, S1y = 0.f, S1z = 0.f;
    float Sxx = 0.f, Sxy = 0.f, Sxz = 0.f, Syy = 0.f, Syz = 0.f, Szz = 0.f;
    int cnt = 0;
    for (int cz = z0; cz <= z1; ++cz) {
      const float ez = fmaxf(0.f, fmaxf((float)cz - u[2], u[2] - (float)(cz + 1)));
      for (int cy = y0; cy <= y1; ++cy) {
        const float ey = fmaxf(0.f, fmaxf((float)cy - u[1], u[1] - (float)(cy + 1)));
        const float rest = rc2 - ez * ez - ey * ey;
        int xa = INT_MAX, xb = -1;
        if (rest >= 0.f) {
          const float rx = sqrtf(rest);
          xa = max((int)floorf(u[0] - rx), 0);
          xb = min((int)floorf(u[0] + rx), g.dim[0] - 1);
        }
        xa = __reduce_min_sync(kFull, xa);
        xb = __reduce_max_sync(kFull, xb);
        if (xa > xb) continue;
        // cells xa..xb of one row are consecutive: one range of entries
        const int row = (cz * g.dim[1] + cy) * g.dim[0];
        const int s0 = off[row + xa], s1 = off[row + xb + 1];
        for (int gs = s0 & ~(kDpcaBox - 1); gs < s1; gs += kDpcaBox) {
          const float4 blo = gbox[2 * (gs / kDpcaBox)], bhi = gbox[2 * (gs / kDpcaBox) + 1];
          const float bx = fmaxf(0.f, fmaxf(blo.x - q.x, q.x - bhi.x));
          const float by = fmaxf(0.f, fmaxf(blo.y - q.y, q.y - bhi.y));
          const float bz = fmaxf(0.f, fmaxf(blo.z - q.z, q.z - bhi.z));
          const float b2 = __fadd_rn(__fadd_rn(__fmul_rn(bx, bx), __fmul_rn(by, by)), __fmul_rn(bz, bz));
          if (!__any_sync(kFull, b2 <= r2)) continue;
          const int j0 = max(gs, s0), j1 = min(gs + kDpcaBox, s1);
#pragma unroll 2
          for (int j = j0 + ((sl - j0) & (kDpcaLanes - 1)); j < j1; j += kDpcaLanes) {
            const float4 pj = sorted[j];
            float dx = pj.x - q.x, dy = pj.y - q.y, dz = pj.z - q.z;
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            const bool in = d2 <= r2;
            dx = in ? dx : 0.f;
            dy = in ? dy : 0.f;
            dz = in ? dz : 0.f;
            const float w = in ? approx_rcp(fmaf(approx_sqrt(d2), inv_r, eps_r)) : 0.f;   // R w
            const float wu = w * inv_r;
            const float wx = wu * dx, wy = wu * dy, wz = wu * dz;   // R w y, y = (x_j - x_i) / R
            S0 += w;
            S1x += wx;
            S1y += wy;
            S1z += wz;
            Sxx = fmaf(wx, dx, Sxx);   // R^2 w y y^T: one more 1/R below
            Sxy = fmaf(wx, dy, Sxy);
            Sxz = fmaf(wx, dz, Sxz);
            Syy = fmaf(wy, dy, Syy);
            Syz = fmaf(wy, dz, Syz);
            Szz = fmaf(wz, dz, Szz);
            cnt += in;
          }
        }
      }
    }
    // partial sums of the kDpcaLanes lanes of a point, fixed order
#pragma unroll
    for (int o = 1; o < kDpcaLanes; o <<= 1) {
      S0 += __shfl_xor_sync(kFull, S0, o);
      S1x += __shfl_xor_sync(kFull, S1x, o);
      S1y += __shfl_xor_sync(kFull, S1y, o);
      S1z += __shfl_xor_sync(kFull, S1z, o);
      Sxx += __shfl_xor_sync(kFull, Sxx, o);
      Sxy += __shfl_xor_sync(kFull, Sxy, o);
      Sxz += __shfl_xor_sync(kFull, Sxz, o);
      Syy += __shfl_xor_sync(kFull, Syy, o);
      Syz += __shfl_xor_sync(kFull, Syz, o);
      Szz += __shfl_xor_sync(kFull, Szz, o);
      cnt += __shfl_xor_sync(kFull, cnt, o);
    }
    if (!valid || sl != 0) continue;
    const int i = __float_as_int(q.w);
    float nv[3] = {0.f, 0.f, 0.f};
    if (cnt >= 3) {
      const float inv = 1.f / S0, inv2 = inv * inv_r;
      const float mx = S1x * inv, my = S1y * inv, mz = S1z * inv;
      float a[3][3];
      a[0][0] = fmaf(-mx, mx, Sxx * inv2);
      a[0][1] = a[1][0] = fmaf(-mx, my, Sxy * inv2);
      a[0][2] = a[2][0] = fmaf(-mx, mz, Sxz * inv2);
      a[1][1] = fmaf(-my, my, Syy * inv2);
      a[1][2] = a[2][1] = fmaf(-my, mz, Syz * inv2);
      a[2][2] = fmaf(-mz, mz, Szz * inv2);
      float v[3];
      if (jacobi_min_vector(a, v) > 0.f) {
        nv[0] = v[0];
        nv[1] = v[1];
        nv[2] = v[2];
      }
    }
    normals[3 * (int64_t)i] = nv[0];
    normals[3 * (int64_t)i + 1] = nv[1];
    normals[3 * (int64_t)i + 2] = nv[2];
    if (counts) counts[i] = cnt;
  }
}

__global__ void dpca_zero_counts_kernel(const int* __restrict__ cell_of, int n, int* __restrict__ counts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (cell_of[i] < 0) counts[i] = 0;
}

}  // namespace

int64_t point_grid_cap(int64_t max_points) {
  return std::min<int64_t>(std::max<int64_t>(2 * max_points, 4096), (int64_t)1 << 26);
}

int point_grid_dims(const float* bbox, double cs_min, int64_t n, int64_t cap_ws, PointGrid* g) {
  const int64_t cap = std::min<int64_t>(cap_ws, std::max<int64_t>(2 * n, 4096));
  double ext[3], emax = 0.0;
  for (int a = 0; a < 3; ++a) {
    ext[a] = std::max(0.0, (double)bbox[3 + a] - (double)bbox[a]);
    emax = std::max(emax, ext[a]);
  }
  double cs = std::max(cs_min, emax / kDpcaAxisCells);
  if (!(cs > 0.0)) cs = 1.0;   // a box of one point
  for (;;) {
    int64_t tot = 1;
    for (int a = 0; a < 3; ++a) {
      g->dim[a] = (int)std::min<double>(std::max(1.0, ceil(ext[a] / cs)), (double)kDpcaAxisCells);
      tot *= g->dim[a];
    }
    if (tot <= cap) break;
    cs *= 1.25;
  }
  for (int a = 0; a < 3; ++a) g->lo[a] = bbox[a];
  g->cs = cs;
  g->inv_cs = (float)(1.0 / cs);
  g->ncell = g->dim[0] * g->dim[1] * g->dim[2];
  return g->ncell;
}

int build_point_grid(wgeo_handle* h, const float* points, int n, const float* bbox, double cs_min, bool ordered,
                     float* zero_normals, PointGrid* g, cudaStream_t s) {
  point_grid_dims(bbox, cs_min, n, h->dp_cell_cap, g);
  const int ncell = g->ncell;
  WGEO_CUDA_TRY(cudaMemsetAsync(h->dp_count, 0, sizeof(int) * (size_t)ncell, s));
  WGEO_CUDA_TRY(cudaMemsetAsync(h->dp_cursor, 0, sizeof(int) * ((size_t)ncell + 1), s));
  dpca_bin_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(points, n, *g, h->dp_cell, h->dp_count, zero_normals);
  WGEO_LAUNCH_CHECK();
  int rc = exclusive_scan(h->dp_count, h->dp_off, ncell, h->dp_scan, s);
  if (rc) return rc;
  dpca_scatter_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(points, n, *g, h->dp_cell, h->dp_off, h->dp_cursor,
                                                          ordered ? h->dp_tmp : h->dp_sorted, h->dp_key);
  WGEO_LAUNCH_CHECK();
  if (ordered) {
    dpca_rank_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(h->dp_tmp, h->dp_key, h->dp_cell, h->dp_off,
                                                         h->dp_off + ncell, h->dp_sorted);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

int launch_dpca(wgeo_handle* h, const float* points, int64_t n64, const float* bbox, float radius, float eps,
                float* normals, int* counts, cudaStream_t s) {
  if (n64 == 0) return WGEO_OK;
  const int n = (int)n64;
  PointGrid g;
  // cells of edge R / kDpcaSub: a warp's union of balls is trimmed to whole cells
  int rc = build_point_grid(h, points, n, bbox, (double)radius / kDpcaSub, true, normals, &g, s);
  if (rc) return rc;
  const int ncell = g.ncell;
  const double cs = g.cs;
  dpca_group_box_kernel<<<grid_blocks(div_up(n, 2 * kDpcaBox) * 32, 256), 256, 0, s>>>(
      h->dp_sorted, h->dp_off + ncell, h->dp_gbox);
  WGEO_LAUNCH_CHECK();
  // reach in cells: R / edge, widened by 1e-3 relative and 4e-3 cells for the
  // rounding of cell coordinates (a few 1e-4 cells at 1024 cells per axis) and
  // of the float membership test (R (1 + 3e-7))
  const float reach = (float)(radius / cs * 1.001 + 4e-3);
  dpca_normal_kernel<<<grid_blocks(div_up(n, kDpcaPts) * 32, 128, 152 * 16), 128, 0, s>>>(
      h->dp_sorted, h->dp_off, h->dp_off + ncell, g, h->dp_gbox, h->dp_cursor + ncell, radius, eps / radius, reach,
      normals, counts);
  WGEO_LAUNCH_CHECK();
  if (counts) {
    dpca_zero_counts_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(h->dp_cell, n, counts);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

}  // namespace wgeo
