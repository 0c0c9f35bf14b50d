// Point binning, counting sort by 8^3 tile, and the fused 27-cell normal splat +
// divergence that produces the Poisson right-hand side b.
//
// Central cell (Sec. 2.3, Eq. 25 "central cell"): floor((x - lo) / h) per axis
// with one IEEE double subtraction and one IEEE double division (__dsub_rn /
// __ddiv_rn: no contraction), clamped into the grid.
//
// Splat (Eqs. 23-25): a~ = 1/2 for the central cell, else the product over
// axes of (1/2) max(0, 1 - |x - c_o| / (2h)); alpha = a~ / sum over in-grid
// cells; V_o = sum_i alpha_{o,i} n_i.  Sums are accumulated in 64-bit fixed
// point (2^-36) in shared memory, so the result does not depend on the order
// in which threads add — b is bit-reproducible run to run.
//
// Divergence (Eqs. 22, 26): b_p = sum_axis (F_{p+1/2} - F_{p-1/2}) with face
// value F = (V_p + V_{p+e}) / 2 on interior faces and 0 on domain faces; the
// face sums are exact integers, rounded once to float32.
#include <algorithm>

#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

struct GridParams {
  double lo[3];
  double h;
  int res;
  int ntile;   // tiles per axis
};

__global__ void bin_points_kernel(const float* __restrict__ pts, const float* __restrict__ nrm,
                                  int64_t n, GridParams g, int* __restrict__ pcell,
                                  float4* __restrict__ pfrac, float4* __restrict__ pnrm,
                                  int* __restrict__ tile_count, DevState* st) {
  unsigned int bits = 0;
  float nmax = 0.f;   // largest |normal component| (bounds the splat's fixed-point terms)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float px = pts[3 * i + 0], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    const float nx = nrm[3 * i + 0], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
    const bool fin = isfinite(px) && isfinite(py) && isfinite(pz) && isfinite(nx) &&
                     isfinite(ny) && isfinite(nz);
    if (!fin) {
      bits |= WGEO_STATUS_NONFINITE_INPUT;
      pcell[i] = -1;
      pfrac[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float p3[3] = {px, py, pz};
    int b[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double u = __ddiv_rn(__dsub_rn((double)p3[a], g.lo[a]), g.h);
      if (u < 0.0 || u > (double)g.res) bits |= WGEO_STATUS_POINT_OUTSIDE_BBOX;
      double fl = floor(u);
      fl = fmin(fmax(fl, 0.0), (double)(g.res - 1));
      b[a] = (int)fl;
      f[a] = (float)(u - fl);
    }
    pcell[i] = pack_cell(b[0], b[1], b[2]);
    pfrac[i] = make_float4(f[0], f[1], f[2], 0.f);
    nmax = fmaxf(nmax, fmaxf(fabsf(nx), fmaxf(fabsf(ny), fabsf(nz))));
    if (pnrm) pnrm[i] = make_float4(nx, ny, nz, 0.f);
    const int t = ((b[2] / kSplatTile) * g.ntile + b[1] / kSplatTile) * g.ntile + b[0] / kSplatTile;
    atomicAdd(&tile_count[t], 1);
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  if (bits && (threadIdx.x & 31) == 0) atomicOr(&st->status, bits);
  // non-negative floats order as their bit patterns
  const unsigned nb = __reduce_max_sync(0xffffffffu, __float_as_uint(nmax));
  if ((threadIdx.x & 31) == 0 && nb) atomicMax(&st->nmax_bits, nb);
}

__global__ void scatter_points_kernel(const float* __restrict__ nrm, int64_t n,
                                      const int* __restrict__ pcell, const float4* __restrict__ pfrac,
                                      int ntile, int* __restrict__ cursor, float4* __restrict__ srec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = pcell[i];
    if (c < 0) continue;
    const int t = ((cell_z(c) / kSplatTile) * ntile + cell_y(c) / kSplatTile) * ntile +
                  cell_x(c) / kSplatTile;
    const int pos = atomicAdd(&cursor[t], 1);
    const float4 f = pfrac[i];
    srec[2 * (int64_t)pos] = make_float4(f.x, f.y, f.z, __int_as_float(c));
    srec[2 * (int64_t)pos + 1] = make_float4(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2], 0.f);
  }
}

constexpr int kR = kSplatTile + 2;  // V region edge: tile plus one halo cell per side
constexpr int kList = 4096;          // shared list of the points reaching a tile
// Narrow sums: when a tile's points all sit in one list (no flush; P <= kList
// points, those whose stencil reaches its V region, so every V sum has at
// most P terms), each V sum is kept as two 32-bit words, q = qh 2^20 + ql
// with ql = q mod 2^20 in [0, 2^20) and qh = floor(q / 2^20).  A term is
// q = rint(alpha n_a 2^36) with alpha <= 1, so |q| <= nmax 2^36 and
// |qh| <= nmax 2^16 + 1 (nmax: the largest |normal component| of the
// points).  With P (nmax 2^16 + 1) < 2^31 the qh sum stays within int32, and
// the ql sum below P 2^20 <= 2^32: sum qh 2^20 + sum ql is the int64 sum
// exactly, taken with native 32-bit shared atomics instead of 64-bit ones.
constexpr int kNarrowShift = 20;
constexpr int div_up_c(int a, int b) { return (a + b - 1) / b; }
constexpr int kSplatThreads = kSplatTile * kSplatTile * kSplatTile;   // one per output cell

// The fixed-point value rint(q) of a float q with |q| <= 2^36 as int64, from
// two int32 conversions: qh = trunc(q / 2^16) and ql = q - qh 2^16 are exact
// (|ql| < 2^16; for |q| >= 2^16, q and qh 2^16 are within a factor 2), and
// rint(q) = qh 2^16 + rint(ql) because qh 2^16 is an even integer.  Equal to
// __float2ll_rn(q), without the 64-bit conversion.
__device__ __forceinline__ long long fix_round(float q) {
  const float qh = truncf(q * 0x1p-16f);
  const float ql = fmaf(-qh, 0x1p16f, q);
  return (long long)__float2int_rz(qh) * 65536ll + (long long)__float2int_rn(ql);
}

// Weights of the mass matrix M = {1, 4, 1} / 6 around a cell at coordinate c
// (offset d = -1, 0, +1), the walls mirrored: an outside neighbour's weight
// folds onto the cell itself.
__device__ __forceinline__ int q1_mass_w(int d, int c, int n) {
  if (d < 0) return c > 0 ? 1 : 0;
  if (d > 0) return c < n - 1 ? 1 : 0;
  return 4 + (c == 0 ? 1 : 0) + (c == n - 1 ? 1 : 0);
}

// The active tiles: those with a point in one of their 27 neighbouring
// tiles (themselves included).  Every other tile has V = 0 and b = 0 there,
// which the caller's memset leaves.  Appended in any order (one atomic per
// warp): each tile's b and partial sums depend on the tile alone.
__global__ void splat_tiles_kernel(const int* __restrict__ tile_off, int ntile, int* __restrict__ list,
                                   DevState* __restrict__ st) {
  const int nt3 = ntile * ntile * ntile;
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count: every lane reaches the ballot
  for (int base = blockIdx.x * blockDim.x; base < nt3; base += gridDim.x * blockDim.x) {
    const int t = base + threadIdx.x;
    bool act = false;
    if (t < nt3) {
      const int tx = t % ntile, ty = (t / ntile) % ntile, tz = t / (ntile * ntile);
      for (int nt = 0; nt < 27 && !act; ++nt) {
        const int ux = tx + nt % 3 - 1, uy = ty + (nt / 3) % 3 - 1, uz = tz + nt / 9 - 1;
        if (ux < 0 || uy < 0 || uz < 0 || ux >= ntile || uy >= ntile || uz >= ntile) continue;
        const int u = (uz * ntile + uy) * ntile + ux;
        act = tile_off[u + 1] > tile_off[u];
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned at = 0;
      if (lane == leader) at = atomicAdd(&st->splat_tiles, (unsigned)__popc(m));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (act) list[at + __popc(m & ((1u << lane) - 1u))] = t;
    }
  }
}

// Persistent: each CTA takes active tiles one after another (a counter on the
// device), one thread per output cell of the 8^3 tile.  Q1: the unlumped
// Galerkin right-hand side b' = 12 sum_xi M M (D_xi V_xi) (the scale of the
// solver's integer-weight operator) instead of the face divergence.
template <bool Q1>
__global__ void __launch_bounds__(kSplatThreads) splat_div_kernel(const float4* __restrict__ srec,
                                                        const int* __restrict__ tile_off, int res,
                                                        int ntile, const int* __restrict__ list,
                                                        DevState* __restrict__ st, float* __restrict__ b,
                                                        double* __restrict__ partials) {
  // V sums: 64-bit fixed point, or (narrow, see kNarrowShift) each sum as two
  // 32-bit words over the same memory
  __shared__ long long V[kR * kR * kR * 3];
  int* const VH = reinterpret_cast<int*>(V);
  unsigned* const VL = reinterpret_cast<unsigned*>(V) + kR * kR * kR * 3;
  bool narrow = false;
  const float nmax = __uint_as_float(st->nmax_bits);
  __shared__ double red[32];   // per-warp sums (16 warps x 2)
  __shared__ int s_list[kList];
  __shared__ int s_cnt;
  __shared__ int s_tile;
  __shared__ int s_nb_start[27], s_nb_cnt[27], s_nb_off[28];
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned it = atomicAdd(&st->splat_next, 1u);
      s_tile = it < st->splat_tiles ? list[it] : -1;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile < 0) return;
    const int tx = tile % ntile, ty = (tile / ntile) % ntile, tz = tile / (ntile * ntile);
    const int T0[3] = {tx * kSplatTile, ty * kSplatTile, tz * kSplatTile};
    for (int k = threadIdx.x; k < kR * kR * kR * 3; k += blockDim.x) V[k] = 0;
    if (threadIdx.x == 0) s_cnt = 0;

    // splat one listed point into the V region (sums in 64-bit fixed point)
    auto splat_point = [&](int k) {
      const float4 r0 = srec[2 * (int64_t)k];
      const int c = __float_as_int(r0.w);
      const int bc[3] = {cell_x(c), cell_y(c), cell_z(c)};
      const float4 r1 = srec[2 * (int64_t)k + 1];
      const float fr[3] = {r0.x, r0.y, r0.z};
      const float nn[3] = {r1.x, r1.y, r1.z};
      // per-axis factors for offsets -1, 0, +1: (x - c_o)/h = frac - 1/2 - delta
      float fac[3][3];
      bool ing[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float t = fabsf(fr[a] - 0.5f - (float)(d - 1));
          fac[a][d] = 0.5f * fmaxf(0.f, 1.f - 0.5f * t);
          const int o = bc[a] + d - 1;
          ing[a][d] = (o >= 0) && (o < res);
        }
      }
      float S = 0.f;
#pragma unroll
      for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            if (!(ing[0][dx] && ing[1][dy] && ing[2][dz])) continue;
            const bool centre = (dx == 1 && dy == 1 && dz == 1);
            S += centre ? 0.5f : fac[0][dx] * fac[1][dy] * fac[2][dz];
          }
      const float inv = 1.f / S;
#pragma unroll
      for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            if (!(ing[0][dx] && ing[1][dy] && ing[2][dz])) continue;
            const int lx = bc[0] + dx - 1 - (T0[0] - 1);
            const int ly = bc[1] + dy - 1 - (T0[1] - 1);
            const int lz = bc[2] + dz - 1 - (T0[2] - 1);
            if (lx < 0 || ly < 0 || lz < 0 || lx >= kR || ly >= kR || lz >= kR) continue;
            const bool centre = (dx == 1 && dy == 1 && dz == 1);
            const float alpha = (centre ? 0.5f : fac[0][dx] * fac[1][dy] * fac[2][dz]) * inv;
            const int vi = ((lz * kR + ly) * kR + lx) * 3;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const long long q = fix_round(alpha * nn[a] * (float)kFixScale);
              if (!q) continue;
              if (narrow) {
                atomicAdd(&VL[vi + a], (unsigned)(q & ((1ll << kNarrowShift) - 1)));
                atomicAdd(&VH[vi + a], (int)(q >> kNarrowShift));
              } else {
                atomicAdd((unsigned long long*)&V[vi + a], (unsigned long long)q);
              }
            }
          }
    };
    // the points of the 27 neighbouring tiles whose stencil reaches this tile's
    // V region go to a shared list first (flushed when it could overflow), so
    // the splatting is spread evenly over the block.  The 27 point ranges are
    // walked as one index space (a prefix over their counts), so a block takes
    // ceil(total / blockDim) list rounds rather than one round per tile.
    if (threadIdx.x < 27) {
      const int nt = threadIdx.x;
      const int ux = tx + nt % 3 - 1, uy = ty + (nt / 3) % 3 - 1, uz = tz + nt / 9 - 1;
      int s0 = 0, c = 0;
      if (ux >= 0 && uy >= 0 && uz >= 0 && ux < ntile && uy < ntile && uz < ntile) {
        const int t = (uz * ntile + uy) * ntile + ux;
        s0 = tile_off[t];
        c = tile_off[t + 1] - s0;
      }
      s_nb_start[nt] = s0;
      s_nb_cnt[nt] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int nt = 0; nt < 27; ++nt) {
        s_nb_off[nt] = acc;
        acc += s_nb_cnt[nt];
      }
      s_nb_off[27] = acc;
    }
    __syncthreads();
    const int total = s_nb_off[27];
    narrow = false;   // a flush while listing splats in 64-bit words
    for (int base = 0; base < total; base += blockDim.x) {
      const int q = base + threadIdx.x;
      int k = 0;
      bool rel = false;
      if (q < total) {
        int lo = 0, hi = 26;   // the last range starting at or before q (empty ranges share starts)
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_nb_off[mid] <= q) lo = mid; else hi = mid - 1;
        }
        k = s_nb_start[lo] + (q - s_nb_off[lo]);
        const int c = __float_as_int(srec[2 * (int64_t)k].w);
        const int bc[3] = {cell_x(c), cell_y(c), cell_z(c)};
        rel = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) rel &= (bc[a] >= T0[a] - 2) && (bc[a] <= T0[a] + kSplatTile + 1);
      }
      // one shared atomic per warp for the list slots
      const unsigned m = __ballot_sync(0xffffffffu, rel);
      if (m) {
        const int leader = __ffs(m) - 1;
        int at = 0;
        if (lane == leader) at = atomicAdd(&s_cnt, __popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (rel) s_list[at + __popc(m & ((1u << lane) - 1u))] = k;
      }
      __syncthreads();
      const int cnt = s_cnt;
      __syncthreads();   // every thread has read the count before the next appends
      if (cnt > kList - (int)blockDim.x) {
        for (int r = threadIdx.x; r < cnt; r += blockDim.x) splat_point(s_list[r]);
        __syncthreads();
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
      }
    }
    {
      // the last (usually the only) list: two-word sums when nothing was
      // splatted before it and its terms stay in range (see kNarrowShift)
      const int cnt = s_cnt;
      narrow = total <= kList - (int)blockDim.x && (float)cnt * (nmax * 65536.f + 1.f) < 2.0e9f;
      for (int q = threadIdx.x; q < cnt; q += blockDim.x) splat_point(s_list[q]);
    }
    __syncthreads();
    if (narrow) {
      // the two-word sums back to int64 in place: all words read, then written
      constexpr int kPer = div_up_c(kR * kR * kR * 3, kSplatThreads);
      long long tmp[kPer];
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int i = threadIdx.x + r * kSplatThreads;
        tmp[r] = i < kR * kR * kR * 3 ? (long long)VH[i] * (1ll << kNarrowShift) + (long long)VL[i] : 0ll;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int i = threadIdx.x + r * kSplatThreads;
        if (i < kR * kR * kR * 3) V[i] = tmp[r];
      }
      __syncthreads();
    }

    const int lx = threadIdx.x % kSplatTile, ly = (threadIdx.x / kSplatTile) % kSplatTile,
              lz = threadIdx.x / (kSplatTile * kSplatTile);
    const int p[3] = {T0[0] + lx, T0[1] + ly, T0[2] + lz};
    float bv = 0.f;
    if (p[0] < res && p[1] < res && p[2] < res) {
      const int l = ((lz + 1) * kR + (ly + 1)) * kR + (lx + 1);
      const int strides[3] = {1, kR, kR * kR};
      long long acc = 0;
      float bf;
      if (!Q1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (p[a] + 1 < res) acc += V[l * 3 + a] + V[(l + strides[a]) * 3 + a];
          if (p[a] - 1 >= 0) acc -= V[(l - strides[a]) * 3 + a] + V[l * 3 + a];
        }
        // acc * 2^-37 rounded once to float (the int64 -> float conversion
        // rounds, the power-of-two scale is exact)
        bf = __ll2float_rn(acc) * (float)kFixInv2;
      } else {
        // 36 sum_xi M M (D_xi V_xi) in exact integer arithmetic: integer mass
        // weights on the two transverse axes around each face difference
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int ab = a == 0 ? 1 : 0, ac = a == 2 ? 1 : 2;
          for (int db = -1; db <= 1; ++db) {
            const int wb = q1_mass_w(db, p[ab], res);
            if (!wb) continue;
            for (int dc = -1; dc <= 1; ++dc) {
              const int wc = q1_mass_w(dc, p[ac], res);
              if (!wc) continue;
              const int lq = l + db * strides[ab] + dc * strides[ac];
              long long d = 0;
              if (p[a] + 1 < res) d += V[lq * 3 + a] + V[(lq + strides[a]) * 3 + a];
              if (p[a] - 1 >= 0) d -= V[(lq - strides[a]) * 3 + a] + V[lq * 3 + a];
              acc += (long long)(wb * wc) * d;
            }
          }
        }
        // 12 b27 = acc * 2^-37 / 3, rounded once to float
        bf = (float)((double)acc * (kFixInv2 / 3.0));
      }
      b[((int64_t)p[2] * res + p[1]) * res + p[0]] = bf;
      bv = bf;
    }
    // sums of b and b^2: float within a warp, FP64 across the warps (fixed order)
    float w1 = bv, w2 = bv * bv;
    for (int o = 16; o > 0; o >>= 1) {
      w1 += __shfl_xor_sync(0xffffffffu, w1, o);
      w2 += __shfl_xor_sync(0xffffffffu, w2, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[2 * (threadIdx.x >> 5)] = (double)w1;
      red[2 * (threadIdx.x >> 5) + 1] = (double)w2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s1 = 0.0, s2 = 0.0;
      for (int q = 0; q < 16; ++q) {
        s1 += red[2 * q];
        s2 += red[2 * q + 1];
      }
      partials[2 * (int64_t)tile] = s1;
      partials[2 * (int64_t)tile + 1] = s2;
    }
  }
}

// Reduces the per-tile partial sums in a fixed order: mean(b) and ||b - mean||.
__global__ void b_stats_kernel(const double* __restrict__ partials, int ntiles, int64_t N,
                               DevState* st) {
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < ntiles; i += blockDim.x) {
    s1 += partials[2 * i];
    s2 += partials[2 * i + 1];
  }
  s1 = block_sum<1024>(s1, red);
  s2 = block_sum<1024>(s2, red);
  if (threadIdx.x == 0) {
    const double mean = s1 / (double)N;
    st->fwd.bmean = mean;
    st->fwd.bmean32 = (float)mean;
    st->fwd.bnorm = sqrt(fmax(s2 - s1 * mean, 0.0));
  }
}

__global__ void unpack_bins_kernel(const int* __restrict__ pcell, int64_t n, int* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = pcell[i];
    out[3 * i] = c < 0 ? -1 : cell_x(c);
    out[3 * i + 1] = c < 0 ? -1 : cell_y(c);
    out[3 * i + 2] = c < 0 ? -1 : cell_z(c);
  }
}

}  // namespace

int launch_unpack_bins(wgeo_handle* h, int* out, cudaStream_t s) {
  if (h->npts == 0) return WGEO_OK;
  unpack_bins_kernel<<<grid_blocks(h->npts, 256), 256, 0, s>>>(h->pcell, h->npts, out);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

int launch_bin_sort_splat(wgeo_handle* h, const float* points, const float* normals, int64_t n,
                          int res, cudaStream_t s) {
  GridParams g;
  for (int a = 0; a < 3; ++a) g.lo[a] = h->lo[a];
  g.h = h->h;
  g.res = res;
  g.ntile = div_up(res, kSplatTile);
  const int ntiles = g.ntile * g.ntile * g.ntile;
  WGEO_CUDA_TRY(cudaMemsetAsync(h->tile_count, 0, sizeof(int) * (ntiles + 1), s));
  if (n > 0) {
    bin_points_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(points, normals, n, g, h->pcell, h->pfrac,
                                                          h->opt.keep_for_backward ? h->pnrm : nullptr,
                                                          h->tile_count, h->dstate);
    WGEO_LAUNCH_CHECK();
  }
  int rc = exclusive_scan(h->tile_count, h->tile_off, ntiles, h->scan_tmp, s);
  if (rc) return rc;
  if (n > 0) {
    WGEO_CUDA_TRY(cudaMemcpyAsync(h->tile_cursor, h->tile_off, sizeof(int) * ntiles,
                                  cudaMemcpyDeviceToDevice, s));
    scatter_points_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(normals, n, h->pcell, h->pfrac, g.ntile,
                                                              h->tile_cursor, h->srec);
    WGEO_LAUNCH_CHECK();
  }
  // b = 0 and zero partial sums outside the active tiles; the tile list
  // reuses the scatter cursors
  WGEO_CUDA_TRY(cudaMemsetAsync(h->b32, 0, sizeof(float) * (size_t)res * res * res, s));
  WGEO_CUDA_TRY(cudaMemsetAsync(h->partials, 0, sizeof(double) * 2 * (size_t)ntiles, s));
  WGEO_CUDA_TRY(cudaMemsetAsync(&h->dstate->splat_tiles, 0, 2 * sizeof(unsigned), s));
  if (n > 0) {
    int* list = h->tile_cursor;
    splat_tiles_kernel<<<grid_blocks(ntiles, 256, h->num_sms * 8), 256, 0, s>>>(h->tile_off, g.ntile, list,
                                                                                 h->dstate);
    WGEO_LAUNCH_CHECK();
    // resident CTAs per SM of each variant (one sm_103a build: the same on every device)
    static std::atomic<int> per_sm[2] = {{0}, {0}};
    const int v = h->opt.galerkin ? 1 : 0;
    int nb = per_sm[v].load(std::memory_order_relaxed);
    if (!nb) {
      const cudaError_t e = v ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, splat_div_kernel<true>, kSplatThreads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, splat_div_kernel<false>, kSplatThreads, 0);
      if (e != cudaSuccess) return WGEO_ERR_CUDA;
      nb = nb > 0 ? nb : 1;
      per_sm[v].store(nb, std::memory_order_relaxed);
    }
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)h->num_sms * nb);
    if (v)
      splat_div_kernel<true><<<grid, kSplatThreads, 0, s>>>(h->srec, h->tile_off, res, g.ntile, list, h->dstate, h->b32,
                                                  h->partials);
    else
      splat_div_kernel<false><<<grid, kSplatThreads, 0, s>>>(h->srec, h->tile_off, res, g.ntile, list, h->dstate, h->b32,
                                                   h->partials);
    WGEO_LAUNCH_CHECK();
  }
  b_stats_kernel<<<1, 1024, 0, s>>>(h->partials, ntiles, (int64_t)res * res * res, h->dstate);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

}  // namespace wgeo
