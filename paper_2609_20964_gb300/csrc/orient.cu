// Parity-based normal orientation (Sec. 2.2): detection radius r_d from the
// largest nearest-neighbour gap (Eqs. baseline_detection_radius and
// expanded_detection_radius), probe rays y_m = x_i + m ds u_i with ds = r_d
// and u_i the normal scaled to unit length, the detection array d_m (some
// point within r_d of y_m), the crossing number N_i (1 -> 0 transitions minus
// the first block, Eq. N_i_define), the leading block length N_one, and the
// three refinement iterations (parity; N_i != 0 or N_one > N_tol; fewer
// crossings than the opposite direction).  Only signs change, so the patterns
// along +u_i and -u_i settle all three iterations.
//
// Every integer decision is taken in float32 with each operation rounded and
// no contraction: squared distances ((dx^2 + dy^2) + dz^2), probe coordinates
// x + (m ds) u, r_{d,0} = 0.5 sqrt(max d2), r_d = gamma r_{d,0}, and the exit
// of the probes from the cloud's bounding box widened by r_d.
//
// GPU layout.  The points are grouped in a cell grid over the box (cell edge
// from the cloud's mean spacing); nearest neighbours come from a shell-by-
// shell search with a stopping bound, one thread per point; a ray is cast by
// one warp, its lanes taking 32 consecutive probes, the detection bits
// gathered with a ballot and the transitions counted with bit operations.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxProbes = 1 << 24;   // m stays exact in float32; rays are cut there

// Order-preserving map of floats to unsigned integers (for atomic min / max).
__device__ __forceinline__ unsigned f2o(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ float d2_rn(float dx, float dy, float dz) {
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// scal: [0..2] ordered min corner, [3..5] ordered max corner of the finite
// points, [6] max over points of the squared nearest-neighbour distance.
__global__ void orient_bounds_kernel(const float4* __restrict__ sorted, const int* __restrict__ total,
                                     unsigned* __restrict__ scal) {
  const int m = *total;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const float4 v = sorted[k];
    lo[0] = fminf(lo[0], v.x), lo[1] = fminf(lo[1], v.y), lo[2] = fminf(lo[2], v.z);
    hi[0] = fmaxf(hi[0], v.x), hi[1] = fmaxf(hi[1], v.y), hi[2] = fmaxf(hi[2], v.z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(kFull, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(kFull, hi[a], o));
    }
  if ((threadIdx.x & 31) == 0 && lo[0] <= hi[0]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&scal[a], f2o(lo[a]));
      atomicMax(&scal[3 + a], f2o(hi[a]));
    }
  }
}

// Nearest other point of every point, shell by shell around its cell: after
// shell k every cell within Chebyshev distance k is done, and a point in any
// other cell lies at least (gap - 1e-3) cells away, gap = the distance from
// the point (in cell units, clamped into the grid) to the faces of the done
// block that have cells beyond them.  The margin covers the rounding of cell
// coordinates.  The maximum of the squared distances goes to scal[6].
__global__ void orient_nn_kernel(const float4* __restrict__ sorted, const int* __restrict__ off,
                                 const int* __restrict__ total, PointGrid g, unsigned* __restrict__ scal) {
  const int m = *total;
  const float cs = (float)g.cs;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const float4 q = sorted[k];
    const int self = __float_as_int(q.w);
    int c[3];
    grid_cell3(g, q.x, q.y, q.z, c);
    const float p[3] = {q.x, q.y, q.z};
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = fminf(fmaxf((p[a] - g.lo[a]) * g.inv_cs, 0.f), (float)g.dim[a]);
    float best = INFINITY;
    for (int sh = 0;; ++sh) {
      for (int dz = -sh; dz <= sh; ++dz) {
        const int cz = c[2] + dz;
        if (cz < 0 || cz >= g.dim[2]) continue;
        for (int dy = -sh; dy <= sh; ++dy) {
          const int cy = c[1] + dy;
          if (cy < 0 || cy >= g.dim[1]) continue;
          const int row = (cz * g.dim[1] + cy) * g.dim[0];
          const bool full = (dz == -sh || dz == sh || dy == -sh || dy == sh);
          // the shell's cells of this row: the whole x run, or its two ends
          for (int part = 0; part < (full ? 1 : 2); ++part) {
            int xa, xb;
            if (full) {
              xa = max(c[0] - sh, 0), xb = min(c[0] + sh, g.dim[0] - 1);
            } else {
              xa = xb = part == 0 ? c[0] - sh : c[0] + sh;
              if (xa < 0 || xa >= g.dim[0]) continue;
            }
            const int s1 = off[row + xb + 1];
            for (int j = off[row + xa]; j < s1; ++j) {
              const float4 pj = sorted[j];
              if (__float_as_int(pj.w) == self) continue;
              best = fminf(best, d2_rn(pj.x - q.x, pj.y - q.y, pj.z - q.z));
            }
          }
        }
      }
      float gap = INFINITY;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (c[a] - sh > 0) gap = fminf(gap, u[a] - (float)(c[a] - sh));
        if (c[a] + sh + 1 < g.dim[a]) gap = fminf(gap, (float)(c[a] + sh + 1) - u[a]);
      }
      if (gap == INFINITY) break;   // every cell searched
      const float reach = fmaxf(gap - 1e-3f, 0.f) * cs;
      if (best <= reach * reach) break;
    }
    if (best < INFINITY) atomicMax(&scal[6], __float_as_uint(best));   // non-negative: bits order
  }
}

struct RayStats {
  int n;     // N (crossings after the first block)
  int one;   // N_one (leading ones)
};

// Whether some point lies within rd of y (float32 test).
__device__ __forceinline__ bool detect(const float4* __restrict__ sorted, const int* __restrict__ off,
                                       const PointGrid& g, float rcell, float rd2, float y0, float y1, float y2) {
  const float y[3] = {y0, y1, y2};
  int a0[3], a1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float uc = fminf(fmaxf((y[a] - g.lo[a]) * g.inv_cs, 0.f), (float)g.dim[a]);
    a0[a] = max((int)floorf(uc - rcell), 0);
    a1[a] = min((int)floorf(uc + rcell), g.dim[a] - 1);
  }
  for (int cz = a0[2]; cz <= a1[2]; ++cz)
    for (int cy = a0[1]; cy <= a1[1]; ++cy) {
      const int row = (cz * g.dim[1] + cy) * g.dim[0];
      const int s1 = off[row + a1[0] + 1];
      for (int j = off[row + a0[0]]; j < s1; ++j) {
        const float4 pj = sorted[j];
        if (d2_rn(pj.x - y0, pj.y - y1, pj.z - y2) <= rd2) return true;
      }
    }
  return false;
}

// One ray cast by a whole warp: (N, N_one) of the detection array along
// x + m ds u, m = 0, 1, ..., ending at the first probe outside [lo_e, hi_e].
__device__ RayStats cast_ray(const float4* __restrict__ sorted, const int* __restrict__ off, const PointGrid& g,
                             float rcell, float rd2, float ds, const float x[3], const float u[3],
                             const float lo_e[3], const float hi_e[3]) {
  const int lane = threadIdx.x & 31;
  int n_all = 0, n_one = -1;
  unsigned prev = 0u;   // d of the previous batch's last probe (none before m = 0)
  for (int base = 0; base < kMaxProbes; base += 32) {
    const float t = __fmul_rn((float)(base + lane), ds);
    float y[3];
    bool outside = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      y[a] = __fadd_rn(x[a], __fmul_rn(t, u[a]));
      outside |= (y[a] < lo_e[a]) || (y[a] > hi_e[a]);
    }
    const bool d = !outside && detect(sorted, off, g, rcell, rd2, y[0], y[1], y[2]);
    const unsigned out_mask = __ballot_sync(kFull, outside);
    unsigned dm = __ballot_sync(kFull, d);
    // the array ends at the first outside probe (its bit is 0)
    const unsigned valid = out_mask ? (0xffffffffu >> (31 - (__ffs(out_mask) - 1))) : 0xffffffffu;
    dm &= valid;
    const unsigned before = (dm << 1) | prev;   // bit p: d of probe p - 1
    n_all += __popc(before & ~dm & valid);
    if (n_one < 0) {
      const unsigned zeros = ~dm & valid;
      if (zeros) n_one = base + __ffs(zeros) - 1;
    }
    prev = dm >> 31;
    if (out_mask) break;
  }
  if (n_one < 0) n_one = kMaxProbes;
  return RayStats{n_all - 1, n_one};
}

// One warp per point (sorted order, chunks from a counter): both rays, the
// three iterations, the flip and the statistics.
__global__ void __launch_bounds__(128, 8) orient_ray_kernel(const float4* __restrict__ sorted,
                                                         const int* __restrict__ off, const int* __restrict__ total,
                                                         PointGrid g, const unsigned* __restrict__ scal, float gamma,
                                                         int n_tol, int* __restrict__ next, float* __restrict__ normals,
                                                         int* __restrict__ stats, float* __restrict__ rd_out) {
  const int m = *total;
  const int lane = threadIdx.x & 31;
  const float r0 = 0.5f * __fsqrt_rn(__uint_as_float(scal[6]));
  const float rd = __fmul_rn(gamma, r0);
  if (rd_out && blockIdx.x == 0 && threadIdx.x == 0) *rd_out = rd;
  const float rd2 = __fmul_rn(rd, rd);
  const float rcell = rd * g.inv_cs * 1.001f + 4e-3f;
  float lo_e[3], hi_e[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo_e[a] = __fsub_rn(o2f(scal[a]), rd);
    hi_e[a] = __fadd_rn(o2f(scal[3 + a]), rd);
  }
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(next, 1);
    k = __shfl_sync(kFull, k, 0);
    if (k >= m) break;
    const float4 q = sorted[k];
    const int i = __float_as_int(q.w);
    const float n0 = normals[3 * (int64_t)i], n1 = normals[3 * (int64_t)i + 1], n2 = normals[3 * (int64_t)i + 2];
    const float ss = d2_rn(n0, n1, n2);
    int st[5] = {0, 0, 0, 0, 0};
    if (rd > 0.f && ss > 0.f && ss < INFINITY) {
      const float len = __fsqrt_rn(ss);
      const float up[3] = {__fdiv_rn(n0, len), __fdiv_rn(n1, len), __fdiv_rn(n2, len)};
      const float um[3] = {-up[0], -up[1], -up[2]};
      const float x[3] = {q.x, q.y, q.z};
      const RayStats p = cast_ray(sorted, off, g, rcell, rd2, rd, x, up, lo_e, hi_e);
      const RayStats mi = cast_ray(sorted, off, g, rcell, rd2, rd, x, um, lo_e, hi_e);
      int s = 1, flags = 0;
      if (p.n & 1) s = -s, flags |= 1;                                        // iteration 0
      const RayStats cur = s > 0 ? p : mi;
      if (cur.n != 0 || cur.one > n_tol) s = -s, flags |= 2;                  // iteration 1
      const RayStats c2 = s > 0 ? p : mi, o2 = s > 0 ? mi : p;
      if (c2.n > o2.n) s = -s, flags |= 4;                                    // iteration 2
      if (s < 0) {
        flags |= 8;
        if (lane == 0) {
          normals[3 * (int64_t)i] = -n0;
          normals[3 * (int64_t)i + 1] = -n1;
          normals[3 * (int64_t)i + 2] = -n2;
        }
      }
      st[0] = p.n, st[1] = p.one, st[2] = mi.n, st[3] = mi.one, st[4] = flags;
    }
    if (stats && lane == 0)
#pragma unroll
      for (int c = 0; c < 5; ++c) stats[5 * (int64_t)i + c] = st[c];
  }
}

// Statistics of points that joined no cell (non-finite): zero.
__global__ void orient_zero_stats_kernel(const int* __restrict__ cell_of, int n, int* __restrict__ stats) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (cell_of[i] < 0)
#pragma unroll
      for (int c = 0; c < 5; ++c) stats[5 * (int64_t)i + c] = 0;
}

}  // namespace

int launch_orient(wgeo_handle* h, const float* points, int64_t n64, const float* bbox, float gamma, int n_tol,
                  float* normals, int* stats, float* rd_out, cudaStream_t s) {
  if (n64 == 0) {
    if (rd_out) WGEO_CUDA_TRY(cudaMemsetAsync(rd_out, 0, sizeof(float), s));
    return WGEO_OK;
  }
  const int n = (int)n64;
  // cell edge: the mean spacing of n points over the box's volume (flat
  // boxes count their thin sides at 1/1024 of the largest)
  double emax = 0.0, vol = 1.0;
  for (int a = 0; a < 3; ++a) emax = std::max(emax, (double)bbox[3 + a] - (double)bbox[a]);
  for (int a = 0; a < 3; ++a) vol *= std::max((double)bbox[3 + a] - (double)bbox[a], emax / kDpcaAxisCells);
  PointGrid g;
  int rc = build_point_grid(h, points, n, bbox, cbrt(vol / n), false, nullptr, &g, s);
  if (rc) return rc;
  const int* total = h->dp_off + g.ncell;
  unsigned* scal = h->or_scal;
  WGEO_CUDA_TRY(cudaMemsetAsync(scal, 0xff, 3 * sizeof(unsigned), s));
  WGEO_CUDA_TRY(cudaMemsetAsync(scal + 3, 0, 4 * sizeof(unsigned), s));
  orient_bounds_kernel<<<grid_blocks(n, 256, 152 * 4), 256, 0, s>>>(h->dp_sorted, total, scal);
  WGEO_LAUNCH_CHECK();
  orient_nn_kernel<<<grid_blocks(n, 128, 152 * 16), 128, 0, s>>>(h->dp_sorted, h->dp_off, total, g, scal);
  WGEO_LAUNCH_CHECK();
  orient_ray_kernel<<<grid_blocks((int64_t)n * 32, 128, 152 * 16), 128, 0, s>>>(
      h->dp_sorted, h->dp_off, total, g, scal, gamma, n_tol, h->dp_cursor + g.ncell, normals, stats, rd_out);
  WGEO_LAUNCH_CHECK();
  if (stats) {
    orient_zero_stats_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(h->dp_cell, n, stats);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

}  // namespace wgeo
