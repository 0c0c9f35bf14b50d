// Iso-value (Sec. 2.4, Eq. 27), marching cubes (Eq. 28), exact signed distance
// to the triangles (Eqs. 29-34) and stencil normals (after Eq. 32).
//
// Iso-value: c = mean over the finite input points of chi interpolated
// trilinearly between cell centres (positions clamped into the node hull),
// accumulated in FP64 with a fixed-order two-pass reduction.
//
// Marching cubes on the (res-1)^3 cubes between cell centres; a node is inside
// iff chi < c.  Cubes are processed in 4^3 bricks (one CTA each): a count pass,
// a scan over bricks, and an emit pass that writes each brick's triangles
// contiguously.  Each triangle stores its three vertices and the global ids of
// the edges they sit on (3 * linear index of the lower node + axis).  A shared
// edge's vertex is computed from the same two chi values by every cube, so it
// is bit-identical across cubes (watertight).
//
// The case table is derived at load time from the face-consistent rule: on a
// face with four crossed edges every inside corner is cut off by its own
// segment; segments are directed with the inside corners on their right seen
// from outside the cube, chained into loops (listed by smallest edge id) and
// fanned from their first edge, so triangles face from inside to outside.
//
// Distance: exact minimum over all triangles of the point-to-triangle distance
// (closest point by Voronoi regions of the triangle: vertices, edges, face —
// the method of Ericson, Real-Time Collision Detection, 5.1.5), found by a
// depth-first, nearest-child-first traversal of an implicit octree of brick
// bounding boxes, pruned only by exact box lower bounds.  Sign: +1 where
// chi >= c, -1 where chi < c (the marching-cubes surface separates the two node
// classes, so this is the parity of crossings of any ray from the node).
#include <math.h>

#include <algorithm>

#include "wgeo_internal.cuh"

namespace wgeo {

__constant__ int c_mc_count[256];
__constant__ signed char c_mc_tris[256][kMaxTriPerCube][3];

// ---------------------------------------------------------------- host: table
namespace {

struct EdgeGeo {
  int axis;
  int c0, c1;  // lower / upper corner
};

void corner_xyz(int k, double* p) {
  p[0] = k & 1;
  p[1] = (k >> 1) & 1;
  p[2] = (k >> 2) & 1;
}

EdgeGeo edge_geo(int e) {
  EdgeGeo g;
  g.axis = e / 4;
  const int a = e % 4;
  int lo[3] = {0, 0, 0};
  const int o0 = (g.axis == 0) ? 1 : 0;
  const int o1 = (g.axis == 2) ? 1 : 2;
  lo[o0] = a & 1;
  lo[o1] = a >> 1;
  g.c0 = lo[0] + 2 * lo[1] + 4 * lo[2];
  lo[g.axis] = 1;
  g.c1 = lo[0] + 2 * lo[1] + 4 * lo[2];
  return g;
}

int table_for_case(int cs, int tris[kMaxTriPerCube * 2][3]) {
  bool in[8];
  for (int k = 0; k < 8; ++k) in[k] = (cs >> k) & 1;
  bool crossed[12];
  for (int e = 0; e < 12; ++e) {
    EdgeGeo g = edge_geo(e);
    crossed[e] = in[g.c0] != in[g.c1];
  }
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  for (int axis = 0; axis < 3; ++axis) {
    for (int side = 0; side < 2; ++side) {
      double nrm[3] = {0, 0, 0};
      nrm[axis] = side ? 1.0 : -1.0;
      int fe[4], nfe = 0;
      for (int e = 0; e < 12; ++e) {
        EdgeGeo g = edge_geo(e);
        double p0[3];
        corner_xyz(g.c0, p0);
        if (g.axis != axis && (int)p0[axis] == side && crossed[e]) fe[nfe++] = e;
      }
      auto mid = [](int e, double* m) {
        EdgeGeo g = edge_geo(e);
        double a[3], b[3];
        corner_xyz(g.c0, a);
        corner_xyz(g.c1, b);
        for (int i = 0; i < 3; ++i) m[i] = 0.5 * (a[i] + b[i]);
      };
      auto add_seg = [&](int a, int b, const double* ref) {
        double pa[3], pb[3];
        mid(a, pa);
        mid(b, pb);
        const double d[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        const double left[3] = {nrm[1] * d[2] - nrm[2] * d[1], nrm[2] * d[0] - nrm[0] * d[2],
                                nrm[0] * d[1] - nrm[1] * d[0]};
        double s = 0;
        for (int i = 0; i < 3; ++i) s += left[i] * (ref[i] - 0.5 * (pa[i] + pb[i]));
        if (s > 0) std::swap(a, b);
        next[a] = b;
      };
      if (nfe == 2) {
        double ref[3] = {0, 0, 0};
        int cnt = 0;
        for (int k = 0; k < 8; ++k) {
          double p[3];
          corner_xyz(k, p);
          if ((int)p[axis] == side && in[k]) {
            for (int i = 0; i < 3; ++i) ref[i] += p[i];
            ++cnt;
          }
        }
        for (int i = 0; i < 3; ++i) ref[i] /= cnt;
        add_seg(fe[0], fe[1], ref);
      } else if (nfe == 4) {
        for (int k = 0; k < 8; ++k) {
          double p[3];
          corner_xyz(k, p);
          if ((int)p[axis] != side || !in[k]) continue;
          int adj[2], na = 0;
          for (int q = 0; q < 4; ++q) {
            EdgeGeo g = edge_geo(fe[q]);
            if (g.c0 == k || g.c1 == k) adj[na++] = fe[q];
          }
          add_seg(adj[0], adj[1], p);
        }
      }
    }
  }
  int nt = 0;
  bool seen[12] = {false};
  for (int e = 0; e < 12; ++e) {
    if (!crossed[e] || seen[e]) continue;
    int loop[12], nl = 0;
    int f = e;
    do {
      loop[nl++] = f;
      seen[f] = true;
      f = next[f];
    } while (f != e && f >= 0 && nl < 12);
    for (int k = 1; k + 1 < nl; ++k) {
      tris[nt][0] = loop[0];
      tris[nt][1] = loop[k];
      tris[nt][2] = loop[k + 1];
      ++nt;
    }
  }
  return nt;
}

}  // namespace

void host_mc_table(int* counts, int* tris) {
  for (int cs = 0; cs < 256; ++cs) {
    int t[kMaxTriPerCube * 2][3];
    const int nt = table_for_case(cs, t);
    counts[cs] = nt;
    for (int k = 0; k < kMaxTriPerCube; ++k)
      for (int v = 0; v < 3; ++v) tris[(cs * kMaxTriPerCube + k) * 3 + v] = (k < nt) ? t[k][v] : -1;
  }
}

int upload_mc_table() {
  int counts[256];
  int tris[256 * kMaxTriPerCube * 3];
  host_mc_table(counts, tris);
  signed char t8[256 * kMaxTriPerCube * 3];
  for (int i = 0; i < 256 * kMaxTriPerCube * 3; ++i) t8[i] = (signed char)tris[i];
  for (int i = 0; i < 256; ++i)
    if (counts[i] > kMaxTriPerCube) return WGEO_ERR_INVALID_ARG;
  WGEO_CUDA_TRY(cudaMemcpyToSymbol(c_mc_count, counts, sizeof(counts)));
  WGEO_CUDA_TRY(cudaMemcpyToSymbol(c_mc_tris, t8, sizeof(t8)));
  return WGEO_OK;
}

// ---------------------------------------------------------------- device
namespace {

struct SurfParams {
  double lo[3];
  double h;
  int res;
  int nb;        // bricks per axis
};

__device__ __forceinline__ int64_t lin3(int i, int j, int k, int n) {
  return ((int64_t)k * n + j) * n + i;
}

__global__ void isovalue_kernel(const float* __restrict__ pts, int64_t n, const int* __restrict__ pcell,
                                const float* __restrict__ chi, SurfParams g,
                                double* __restrict__ partials) {
  __shared__ double red[32];
  double s = 0.0, cnt = 0.0;
  const int res = g.res;
  // lo and 1/h as float-float pairs: the cells and weights come from
  // node_coord_ff, the FP64 pipe only sums
  float lo_hi[3], lo_lo[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo_hi[a] = (float)g.lo[a];
    lo_lo[a] = (float)(g.lo[a] - (double)lo_hi[a]);
  }
  const double ih = 1.0 / g.h;
  const float ih_hi = (float)ih, ih_lo = (float)(ih - (double)ih_hi);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (pcell[i] < 0) continue;
    int i0[3];
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      node_cell_ff(node_coord_ff(pts[3 * i + a], lo_hi[a], lo_lo[a], ih_hi, ih_lo), res, i0[a], t[a]);
    // the interpolated value in float-float (weights and products in float)
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
      const float w = (dx ? t[0] : 1.f - t[0]) * (dy ? t[1] : 1.f - t[1]) * (dz ? t[2] : 1.f - t[2]);
      v = ff_add_f(v, w * chi[lin3(i0[0] + dx, i0[1] + dy, i0[2] + dz, res)]);
    }
    s += (double)v.x + (double)v.y;
    cnt += 1.0;
  }
  s = block_sum<256>(s, red);
  cnt = block_sum<256>(cnt, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s;
    partials[2 * blockIdx.x + 1] = cnt;
  }
}

__global__ void isovalue_finalize_kernel(const double* __restrict__ partials, int nblocks, DevState* st) {
  __shared__ double red[32];
  double s = 0.0, cnt = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    s += partials[2 * i];
    cnt += partials[2 * i + 1];
  }
  s = block_sum<1024>(s, red);
  cnt = block_sum<1024>(cnt, red);
  if (threadIdx.x == 0) {
    st->c = cnt > 0.0 ? s / cnt : 0.0;
    float cu = (float)st->c;
    if ((double)cu < st->c) cu = nextafterf(cu, INFINITY);
    st->c_up = cu;
    st->npts = (long long)cnt;
  }
}

// Case code of a cube: bit q set when corner q is inside (chi < c, tested as
// chi < c_up, the smallest float >= c).
__device__ __forceinline__ int cube_code(const float* __restrict__ chi, int i, int j, int k, int n, float c_up) {
  int code = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float v = chi[lin3(i + (q & 1), j + ((q >> 1) & 1), k + (q >> 2), n)];
    code |= (v < c_up) ? (1 << q) : 0;
  }
  return code;
}

// Cube (i,j,k) of a 4^3 brick handled by thread t: Morton order inside the
// brick, so the 8 cubes of each 2^3 sub-brick (an octree leaf) are the
// contiguous threads 8k..8k+7 and their triangles are contiguous in memory.
__device__ __forceinline__ void brick_cube(int t, int& lx, int& ly, int& lz) {
  lx = (t & 1) | (((t >> 3) & 1) << 1);
  ly = ((t >> 1) & 1) | (((t >> 4) & 1) << 1);
  lz = ((t >> 2) & 1) | (((t >> 5) & 1) << 1);
}

// Inside bits of the nodes (chi < c, tested as chi < c_up), 32 per word
// along x: word w of row (j, k) holds x = 32 w .. 32 w + 31 (bits past the
// grid's edge clear), at bits[(k n + j) nw + w], nw = ceil(n / 32).  One warp
// per word: coalesced reads of chi, one ballot.
constexpr int kBitRows = 8;   // rows per warp in mc_bits_kernel (loads in flight per lane)
__global__ void __launch_bounds__(256) mc_bits_kernel(const float* __restrict__ chi, int n, int nw,
                                                      const DevState* __restrict__ st,
                                                      unsigned* __restrict__ bits) {
  // block (32, 8): warp y takes word blockIdx.x of kBitRows consecutive rows
  // (k n + j), their loads issued together
  const int row0 = (blockIdx.y * 8 + threadIdx.y) * kBitRows;
  const int x = 32 * blockIdx.x + threadIdx.x;
  const float c_up = st->c_up;
  float v[kBitRows];
#pragma unroll
  for (int r = 0; r < kBitRows; ++r)
    v[r] = (x < n && row0 + r < n * n) ? chi[(int64_t)(row0 + r) * n + x] : INFINITY;
#pragma unroll
  for (int r = 0; r < kBitRows; ++r) {
    const unsigned m = __ballot_sync(0xffffffffu, v[r] < c_up);
    if (threadIdx.x == 0 && row0 + r < n * n) bits[(row0 + r) * nw + blockIdx.x] = m;
  }
}

// Four 4^3 bricks of cubes per CTA (consecutive brick indices), 64 threads
// (two warps) per brick.
constexpr int kMcBricks = 4;

// Triangles per 4^3 brick from the inside bits.  A thread takes 32 cubes
// along x (one word) of one cube row: the cube's 8 corner bits are bit b and
// bit b + 1 of the four node rows (j, k), (j + 1, k), (j, k + 1), (j + 1,
// k + 1), so the cubes that the surface crosses (corners neither all inside
// nor all outside) come out of eight word operations, and only those look up
// their case.  The 16 threads of one word and brick row (j, k mod 4) are 16
// consecutive lanes; their counts for the word's 8 bricks are summed by
// shuffles (only where a cube is crossed) and written by the first.
__global__ void mc_count_kernel(const unsigned* __restrict__ bits, SurfParams g, int nw,
                                int* __restrict__ brick_count) {
  const int n = g.res, m = n - 1, nb = g.nb;
  const int cw = (m + 31) / 32;              // cube words per row
  const int64_t groups = (int64_t)cw * nb * nb;
  const int lane = threadIdx.x & 31, sub = lane & 15;
  // warp-uniform trip count (two groups per warp): every lane reaches the shuffles
  for (int64_t wb = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; 2 * wb < groups;
       wb += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t gi = 2 * wb + (lane >> 4);   // (w, by, bz) of this half-warp
    const bool ok = gi < groups;
    const int w = ok ? (int)(gi % cw) : 0;
    const int by = ok ? (int)((gi / cw) % nb) : 0, bz = ok ? (int)(gi / ((int64_t)cw * nb)) : 0;
    const int j = 4 * by + (sub & 3), k = 4 * bz + (sub >> 2);
    // triangle counts of the word's 8 bricks, 16 bits each (at most 320 per
    // brick after the half-warp sum): bricks 0-3 in c03, 4-7 in c47
    unsigned long long c03 = 0ull, c47 = 0ull;
    bool any = false;
    if (ok && j < m && k < m) {
      unsigned A[4], B[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t row = (int64_t)(k + (r >> 1)) * n + (j + (r & 1));
        const unsigned lo = bits[row * nw + w];
        const unsigned hi = (w + 1 < nw) ? bits[row * nw + w + 1] : 0u;
        A[r] = lo;
        B[r] = (lo >> 1) | (hi << 31);
      }
      const unsigned all_in = A[0] & A[1] & A[2] & A[3] & B[0] & B[1] & B[2] & B[3];
      const unsigned all_out = ~(A[0] | A[1] | A[2] | A[3] | B[0] | B[1] | B[2] | B[3]);
      const int xv = m - 32 * w;             // cubes of this word inside the grid
      const unsigned valid = xv >= 32 ? 0xffffffffu : ((1u << xv) - 1u);
      unsigned mixed = ~(all_in | all_out) & valid;
      any = mixed != 0u;
      while (mixed) {
        const int b = __ffs(mixed) - 1;
        mixed &= mixed - 1u;
        // corner q = (x offset q & 1, y offset q >> 1 & 1, z offset q >> 2)
        int code = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const unsigned word = (q & 1) ? B[q >> 1] : A[q >> 1];
          code |= (int)((word >> b) & 1u) << q;
        }
        const unsigned long long add = (unsigned long long)c_mc_count[code] << (16 * ((b >> 2) & 3));
        if (b < 16) c03 += add; else c47 += add;
      }
    }
    // sum over the 16 lanes of the half-warp (both halves take part)
    if (__any_sync(0xffffffffu, any)) {
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        c03 += __shfl_xor_sync(0xffffffffu, c03, o);
        c47 += __shfl_xor_sync(0xffffffffu, c47, o);
      }
    }
    if (ok && sub == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int bx = 8 * w + q;
        const unsigned long long v = q < 4 ? c03 : c47;
        if (bx < nb) brick_count[((int64_t)bz * nb + by) * nb + bx] = (int)((v >> (16 * (q & 3))) & 0xffffull);
      }
    }
  }
}

__global__ void mc_total_kernel(const int* __restrict__ brick_off, int nbricks, int64_t cap,
                                int* __restrict__ leaf_off, DevState* st) {
  const long long T = brick_off[nbricks];
  st->ntris = T;
  leaf_off[8 * (int64_t)nbricks] = brick_off[nbricks];
  if (T > cap) atomicOr(&st->status, WGEO_STATUS_MESH_CAPACITY);
  if (T == 0) atomicOr(&st->status, WGEO_STATUS_EMPTY_SURFACE);
}

__device__ __forceinline__ void edge_lower_offset(int e, int& ox, int& oy, int& oz, int& axis) {
  axis = e >> 2;
  const int a = e & 3;
  int o[3] = {0, 0, 0};
  const int o0 = (axis == 0) ? 1 : 0;
  const int o1 = (axis == 2) ? 1 : 2;
  o[o0] = a & 1;
  o[o1] = a >> 1;
  ox = o[0];
  oy = o[1];
  oz = o[2];
}

// Edges of a brick's cubes, by the local coordinates (0..kBrick) of their
// lower end node: along the edge's axis 0..kBrick-1, across it 0..kBrick.
constexpr int kEdgesPerAxis = kBrick * (kBrick + 1) * (kBrick + 1);
constexpr int kBrickEdges = 3 * kEdgesPerAxis;
constexpr int div_up_c(int a, int b) { return (a + b - 1) / b; }
__device__ __forceinline__ int brick_edge_slot(int ax, int ex, int ey, int ez) {
  const int u = ax == 0 ? ex : (ax == 1 ? ey : ez);   // along the axis
  const int v = ax == 0 ? ey : ex;                     // the first other axis
  const int w = ax == 2 ? ey : ez;                     // the second
  return ax * kEdgesPerAxis + (w * (kBrick + 1) + v) * kBrick + u;
}
__device__ __forceinline__ void brick_edge_of_slot(int sl, int& ax, int& ex, int& ey, int& ez) {
  ax = sl / kEdgesPerAxis;
  const int r = sl - ax * kEdgesPerAxis;
  const int u = r % kBrick, v = (r / kBrick) % (kBrick + 1), w = r / (kBrick * (kBrick + 1));
  ex = ax == 0 ? u : v;
  ey = ax == 1 ? u : (ax == 0 ? v : w);
  ez = ax == 2 ? u : w;
}

// Emits each brick's triangles contiguously (Morton cube order) and the
// triangle offset of each of its 8 sub-bricks (octree leaves).  A vertex is
// placed in FP64 from the cube edge's two indicator values (Eq. 28); with
// `chiff` (the refined float-float indicator, current buffer chosen by the
// solve's index) those values carry the float-float low parts, so the vertex
// follows the refined solution rather than its float32 copy.  tris holds the
// vertices rounded to float32; tris_lo (may be null) their residuals
// (double vertex - float vertex, rounded to float), so that hi + lo keeps
// about 48 bits: near-tie decisions and the adjoint's closest points use it.
// The bricks with triangles, listed (one atomic per warp); an empty brick
// writes its 8 leaf offsets here (all equal to its triangle offset).
__global__ void mc_live_kernel(const int* __restrict__ brick_off, int nbr, int* __restrict__ leaf_off,
                               int* __restrict__ list, unsigned* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count: every lane reaches the ballot
  for (int b0 = blockIdx.x * blockDim.x; b0 < nbr; b0 += gridDim.x * blockDim.x) {
    const int br = b0 + threadIdx.x;
    bool live = false;
    if (br < nbr) {
      const int base = brick_off[br];
      live = brick_off[br + 1] != base;
      if (!live) {
        int4* lo4 = reinterpret_cast<int4*>(leaf_off + 8 * (int64_t)br);
        lo4[0] = make_int4(base, base, base, base);
        lo4[1] = make_int4(base, base, base, base);
      }
    }
    const unsigned mk = __ballot_sync(0xffffffffu, live);
    if (mk) {
      const int leader = __ffs(mk) - 1;
      unsigned at = 0;
      if (lane == leader) at = atomicAdd(count, (unsigned)__popc(mk));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (live) list[at + __popc(mk & ((1u << lane) - 1u))] = br;
    }
  }
}

__global__ void __launch_bounds__(64 * kMcBricks) mc_emit_kernel(const float* __restrict__ chi, ChiFF chiff,
                                                                 SurfParams g, const DevState* __restrict__ st,
                                                                 const int* __restrict__ brick_off, int64_t cap,
                                                                 const int* __restrict__ live_list,
                                                                 const unsigned* __restrict__ nlive,
                                                                 Tri* __restrict__ tris, Tri* __restrict__ tris_lo,
                                                                 int* __restrict__ leaf_off,
                                                                 unsigned* __restrict__ leaf_cnt) {
  const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = g.res, m = n - 1;
  const double c = st->c;
  const float c_up = st->c_up;
  const float2* __restrict__ xff = chiff.p[0] ? chiff.p[st->fwd.xidx] : nullptr;
  __shared__ int wt[2 * kMcBricks];
  // the brick's crossing edges (listed first, so that the FP64 placement
  // runs on full warps), and its vertices, one per crossing edge (hi with
  // the edge id in .w; lo)
  __shared__ short s_cross[kMcBricks][kBrickEdges];
  __shared__ int s_ncross[kMcBricks];
  __shared__ float4 s_vh[kMcBricks][kBrickEdges], s_vl[kMcBricks][kBrickEdges];
  const unsigned count = *nlive;
  // persistent: kMcBricks listed bricks per iteration (the same trip count in
  // the whole CTA: every thread reaches the barriers)
  for (unsigned b0 = blockIdx.x * kMcBricks; b0 < count; b0 += gridDim.x * kMcBricks) {
    const bool live = b0 + grp < count;
    const int br = live ? live_list[b0 + grp] : 0;
    const int base = live ? brick_off[br] : 0;
    const int bx = br % g.nb, by = (br / g.nb) % g.nb, bz = br / (g.nb * g.nb);
    int i = 0, j = 0, k = 0;
    int code = 0, cnt = 0;
    if (live) {
      int lx, ly, lz;
      brick_cube(t, lx, ly, lz);
      i = bx * kBrick + lx;
      j = by * kBrick + ly;
      k = bz * kBrick + lz;
      if (i < m && j < m && k < m) {
        code = cube_code(chi, i, j, k, n, c_up);
        cnt = c_mc_count[code];
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int tt = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += tt;
    }
    // the 8 cubes' triangle counts of each leaf (8 consecutive threads), 4 bits each
    unsigned pk = (unsigned)cnt << (4 * (t & 7));
    pk |= __shfl_xor_sync(0xffffffffu, pk, 1);
    pk |= __shfl_xor_sync(0xffffffffu, pk, 2);
    pk |= __shfl_xor_sync(0xffffffffu, pk, 4);
    if (live && leaf_cnt && (t & 7) == 0) leaf_cnt[8 * (int64_t)br + (t >> 3)] = pk;
    if (lane == 31) wt[w] = incl;
    if (t == 0) s_ncross[grp] = 0;
    __syncthreads();
    if (live) {
      for (int r = 0; r < div_up_c(kBrickEdges, 64); ++r) {   // the same trip count in both warps
        const int e = t + 64 * r;
        bool cross = false;
        if (e < kBrickEdges) {
          int ax, ex, ey, ez;
          brick_edge_of_slot(e, ax, ex, ey, ez);
          const int pi = bx * kBrick + ex, pj = by * kBrick + ey, pk = bz * kBrick + ez;
          if (pi + (ax == 0) < n && pj + (ax == 1) < n && pk + (ax == 2) < n) {
            const int64_t p = lin3(pi, pj, pk, n);
            const int64_t stride = (ax == 0) ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
            // crossing exactly when the two corner bits of the cube codes differ
            cross = (chi[p] < c_up) != (chi[p + stride] < c_up);
          }
        }
        const unsigned mk = __ballot_sync(0xffffffffu, cross);
        if (mk) {
          const int leader = __ffs(mk) - 1;
          int at = 0;
          if (lane == leader) at = atomicAdd(&s_ncross[grp], __popc(mk));
          at = __shfl_sync(0xffffffffu, at, leader);
          if (cross) s_cross[grp][at + __popc(mk & ((1u << lane) - 1u))] = (short)e;
        }
      }
    }
    __syncthreads();
    if (live) {
      const int nc = s_ncross[grp];
      for (int ci = t; ci < nc; ci += 64) {
        const int e = s_cross[grp][ci];
        int ax, ex, ey, ez;
        brick_edge_of_slot(e, ax, ex, ey, ez);
        const int pi = bx * kBrick + ex, pj = by * kBrick + ey, pk = bz * kBrick + ez;
        const int64_t p = lin3(pi, pj, pk, n);
        const int64_t stride = (ax == 0) ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
        double c1, c2;
        if (xff) {
          const float2 f1 = xff[p], f2 = xff[p + stride];
          c1 = (double)f1.x + (double)f1.y;
          c2 = (double)f2.x + (double)f2.y;
        } else {
          c1 = (double)chi[p];
          c2 = (double)chi[p + stride];
        }
        const double eta = (c - c1) / (c2 - c1);
        // node centre, moved by eta h along the edge's axis
        double px = fma(pi + 0.5, g.h, g.lo[0]), py = fma(pj + 0.5, g.h, g.lo[1]), pz = fma(pk + 0.5, g.h, g.lo[2]);
        if (ax == 0) px = fma(eta, g.h, px);
        else if (ax == 1) py = fma(eta, g.h, py);
        else pz = fma(eta, g.h, pz);
        const int gid = (int)(3 * p + ax);
        const float hx = (float)px, hy = (float)py, hz = (float)pz;
        s_vh[grp][e] = make_float4(hx, hy, hz, __int_as_float(gid));
        s_vl[grp][e] = make_float4((float)(px - (double)hx), (float)(py - (double)hy), (float)(pz - (double)hz), 0.f);
      }
    }
    __syncthreads();
    if (live) {
      const int excl = incl - cnt + ((w & 1) ? wt[w - 1] : 0);
      if ((t & 7) == 0) leaf_off[8 * (int64_t)br + (t >> 3)] = base + excl;
      const int li = i - bx * kBrick, lj = j - by * kBrick, lk = k - bz * kBrick;
      for (int q = 0; q < cnt; ++q) {
        const int64_t idx = (int64_t)base + excl + q;
        if (idx >= cap) break;
        auto slot = [&](int v) {
          int ox, oy, oz, ax;
          edge_lower_offset(c_mc_tris[code][q][v], ox, oy, oz, ax);
          return brick_edge_slot(ax, li + ox, lj + oy, lk + oz);
        };
        const int s0 = slot(0), s1 = slot(1), s2 = slot(2);
        tris[idx] = Tri{s_vh[grp][s0], s_vh[grp][s1], s_vh[grp][s2]};
        if (tris_lo) tris_lo[idx] = Tri{s_vl[grp][s0], s_vl[grp][s1], s_vl[grp][s2]};
      }
    }
    __syncthreads();   // the shared arrays are reused by the next bricks
  }
}

// ---- octree of "pucks" over the leaves (2^3-cube sub-bricks).  A puck is a
// solid cylinder (centre c, unit axis n, radius r, half-thickness t) holding
// every vertex of the node's triangles, hence (by convexity) the triangles
// themselves; its exact distance is a lower bound on their distance.  For a
// smooth patch the cylinder is thin and oriented along the surface normal, so
// the bound stays tight even for far, oblique queries.  Empty node: r < 0.
struct PyrInfo {
  int nlev;
  int dim[12];
  long long off[12];
};

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ int leaf_index(int lx, int ly, int lz, int nb) {
  const int br = ((lz >> 1) * nb + (ly >> 1)) * nb + (lx >> 1);
  return 8 * br + ((lx & 1) | ((ly & 1) << 1) | ((lz & 1) << 2));
}

constexpr float kPuckPad = 1e-5f;   // relative inflation: rounding of the bound stays conservative

// 10-bit hash of a marching-cubes vertex (its global edge id).
__device__ __forceinline__ unsigned vertex_hash10(float gid_bits) {
  return (__float_as_uint(gid_bits) * 0x9E3779B1u) >> 22;
}

// Search record of a triangle for the distance search: vertex a and the edge
// vectors ab, ac with the Gram entries |ab|^2 and |ac|^2 (ab.ac is formed
// where it is used), the reciprocals the Voronoi regions divide by (0 for a
// zero-length edge or a collapsed triangle), and in the slot of ab.ac the
// 10-bit hashes of the three vertices (bits 0-9 a, 10-19 b, 20-29 c), which
// name a closest vertex or edge without another memory access.
// With the vertices' low parts (lo, may be null) the edge vectors are the
// float32 roundings of the differences of the ~48-bit vertices, not the
// differences of the float32 vertices: their directions then carry float32
// rounding (~6e-8 relative) instead of the vertices' absolute rounding,
// which a far node's closest point would amplify by distance / edge length.
__device__ __forceinline__ void write_search_record(const Tri& tr, const Tri* lo, float4* __restrict__ rec) {
  const float3 a = f3(tr.a), b = f3(tr.b), c = f3(tr.c);
  float3 ab = sub3(b, a), ac = sub3(c, a), bc = sub3(c, b);
  if (lo) {
    const float3 al = f3(lo->a), bl = f3(lo->b), cl = f3(lo->c);
    ab = make_float3(ab.x + (bl.x - al.x), ab.y + (bl.y - al.y), ab.z + (bl.z - al.z));
    ac = make_float3(ac.x + (cl.x - al.x), ac.y + (cl.y - al.y), ac.z + (cl.z - al.z));
    bc = make_float3(bc.x + (cl.x - bl.x), bc.y + (cl.y - bl.y), bc.z + (cl.z - bl.z));
  }
  const float e00 = dot3(ab, ab), e11 = dot3(ac, ac), ebc = dot3(bc, bc);
  const float3 cr = cross3(ab, ac);
  const float det = dot3(cr, cr);   // = |ab|^2 |ac|^2 - (ab.ac)^2, without the cancellation
  rec[0] = make_float4(a.x, a.y, a.z, e00);
  const unsigned vk = vertex_hash10(tr.a.w) | (vertex_hash10(tr.b.w) << 10) | (vertex_hash10(tr.c.w) << 20);
  rec[1] = make_float4(ab.x, ab.y, ab.z, __uint_as_float(vk));
  rec[2] = make_float4(ac.x, ac.y, ac.z, e11);
  rec[3] = make_float4(e00 > 0.f ? 1.f / e00 : 0.f, e11 > 0.f ? 1.f / e11 : 0.f, ebc > 0.f ? 1.f / ebc : 0.f,
                       det > 0.f ? 1.f / det : 0.f);
}

// Leaf pucks, pass 1 (every leaf): an empty leaf gets the empty puck; a
// leaf with triangles goes to the list of live leaves (one atomic per warp),
// which the fitting passes then take with full warps.
__global__ void puck_leaf_scan_kernel(const int* __restrict__ leaf_off, int nb, int64_t cap,
                                      float4* __restrict__ pyr, int* __restrict__ live, DevState* __restrict__ st) {
  const int nl = 2 * nb;
  const int64_t nleaf = (int64_t)nl * nl * nl;
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count: every lane reaches the ballot
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nleaf; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = base + threadIdx.x;
    bool full = false;
    if (t < nleaf) {
      const int lx = (int)(t % nl), ly = (int)((t / nl) % nl), lz = (int)(t / ((int64_t)nl * nl));
      const int li = leaf_index(lx, ly, lz, nb);
      full = min((int64_t)leaf_off[li + 1], cap) > (int64_t)leaf_off[li];
      if (!full) {
        pyr[2 * t] = make_float4(0.f, 0.f, 0.f, -1.f);
        pyr[2 * t + 1] = make_float4(0.f, 0.f, 1.f, 0.f);
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, full);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned at = 0;
      if (lane == leader) at = atomicAdd(&st->nleaf_live, (unsigned)__popc(m));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (full) live[at + __popc(m & ((1u << lane) - 1u))] = (int)t;
    }
  }
}

// Puck (centre + radius, axis + half-thickness) fitted to the vertices of
// triangles [q0, q1): centroid and mean area normal, then the largest radial
// and axial vertex offsets in that frame, padded so the bound stays
// conservative under float rounding.
__device__ __forceinline__ void fit_puck(const Tri* __restrict__ tris, int64_t q0, int64_t q1, float4& A, float4& B) {
  float3 cs = make_float3(0.f, 0.f, 0.f), ns = make_float3(0.f, 0.f, 0.f);
  for (int64_t q = q0; q < q1; ++q) {
    const Tri tr = tris[q];
    const float3 a = f3(tr.a), b = f3(tr.b), c = f3(tr.c);
    cs.x += a.x + b.x + c.x;
    cs.y += a.y + b.y + c.y;
    cs.z += a.z + b.z + c.z;
    const float3 cr = cross3(sub3(b, a), sub3(c, a));
    ns.x += cr.x;
    ns.y += cr.y;
    ns.z += cr.z;
  }
  const float inv = 1.f / (3.f * (float)(q1 - q0));
  const float3 cc = make_float3(cs.x * inv, cs.y * inv, cs.z * inv);
  const float nn = sqrtf(dot3(ns, ns));
  const float3 nv = nn > 0.f ? make_float3(ns.x / nn, ns.y / nn, ns.z / nn) : make_float3(0.f, 0.f, 1.f);
  float r = 0.f, th = 0.f;
  for (int64_t q = q0; q < q1; ++q) {
    const Tri tr = tris[q];
    const float4 vv[3] = {tr.a, tr.b, tr.c};
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float3 d = sub3(f3(vv[v]), cc);
      const float z = dot3(d, nv);
      const float rho2 = fmaxf(dot3(d, d) - z * z, 0.f);
      th = fmaxf(th, fabsf(z));
      r = fmaxf(r, sqrtf(rho2));
    }
  }
  const float pad = kPuckPad * (fabsf(cc.x) + fabsf(cc.y) + fabsf(cc.z) + r + th) + 1e-7f;
  A = make_float4(cc.x, cc.y, cc.z, r * (1.f + kPuckPad) + pad);
  B = make_float4(nv.x, nv.y, nv.z, th * (1.f + kPuckPad) + pad);
}

// Leaf pucks, pass 2 (live leaves): the triangles' search records, the
// leaf's puck fitted to its vertices, and (cell_pyr non-null) one puck per
// cube of the leaf that holds triangles, stored at the slot of the cube's
// first triangle (cell_pyr[2 q0], [2 q0 + 1]); leaf_cnt packs the cubes'
// triangle counts, 4 bits per cube in the leaf's cube order.
__global__ void puck_leaf_kernel(const Tri* __restrict__ tris, const Tri* __restrict__ tris_lo,
                                 const int* __restrict__ leaf_off, const unsigned* __restrict__ leaf_cnt, int nb,
                                 int64_t cap, const int* __restrict__ live, const DevState* __restrict__ st,
                                 float4* __restrict__ pyr, float4* __restrict__ tris_s,
                                 float4* __restrict__ cell_pyr) {
  const int nl = 2 * nb;
  const int64_t nlive = st->nleaf_live;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nlive;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = live[it];
    const int lx = (int)(t % nl), ly = (int)((t / nl) % nl), lz = (int)(t / ((int64_t)nl * nl));
    const int li = leaf_index(lx, ly, lz, nb);
    const int64_t s0 = leaf_off[li];
    const int64_t s1 = min((int64_t)leaf_off[li + 1], cap);
    for (int64_t q = s0; q < s1; ++q) {
      const Tri tr = tris[q];
      if (tris_lo) {
        const Tri tl = tris_lo[q];
        write_search_record(tr, &tl, tris_s + kTriRec * q);
      } else {
        write_search_record(tr, nullptr, tris_s + kTriRec * q);
      }
    }
    float4 A, B;
    fit_puck(tris, s0, s1, A, B);
    pyr[2 * t] = A;
    pyr[2 * t + 1] = B;
    if (cell_pyr) {
      unsigned cn = leaf_cnt[li];
      int64_t q0 = s0;
      for (; cn != 0u; cn >>= 4) {
        const int64_t q1 = min(q0 + (int64_t)(cn & 15u), s1);
        if (q0 < q1) {
          fit_puck(tris, q0, q1, A, B);
          cell_pyr[2 * q0] = A;
          cell_pyr[2 * q0 + 1] = B;
        }
        q0 += cn & 15u;
      }
    }
  }
}

// Tight puck of an internal node at level l >= 1 (dim d_l; level 1 = bricks):
// axis and centre from its own triangles, radius and half-thickness from
// their vertices (two passes over the bricks it covers).
// Squared distance from p to the solid cylinder of a puck (INF when empty).
__device__ __forceinline__ float puck_dist2(const float3 p, const float4 A, const float4 B) {
  if (A.w < 0.f) return INFINITY;
  const float3 d = make_float3(p.x - A.x, p.y - A.y, p.z - A.z);
  const float z = d.x * B.x + d.y * B.y + d.z * B.z;
  // rho from the hardware reciprocal square root (a few ulp), scaled down by
  // 1e-6 so that it stays below the exact value: a lower bound still
  const float x2 = fmaxf(d.x * d.x + d.y * d.y + d.z * d.z - z * z, 0.f);
  const float rho = x2 * rsqrtf(fmaxf(x2, 1e-30f)) * (1.f - 1e-6f);
  const float dz = fmaxf(fabsf(z) - B.w, 0.f);
  const float dr = fmaxf(rho - A.w, 0.f);
  return dz * dz + dr * dr;
}

// Vertex-fitted pucks for every octree level above the leaves.  A node's
// frame is its vertex centroid and mean area normal; both come from sums
// that add up the tree (per brick first: a level-1 node is one brick).  The
// radius and half-thickness are the largest radial and axial vertex offsets
// in that frame, taken in one pass over the leaves for all levels at once
// (warp-aggregated atomic maxima on the bits of non-negative floats).  Aux
// slots cover the nodes of levels >= 1: aux index = pyramid index - off[1].
__device__ __forceinline__ void node_frame(const float4 s0, const float4 s1, float3& c, float3& ax) {
  const float inv = 1.f / (3.f * s0.w);
  c = make_float3(s0.x * inv, s0.y * inv, s0.z * inv);
  const float nn = sqrtf(s1.x * s1.x + s1.y * s1.y + s1.z * s1.z);
  ax = nn > 0.f ? make_float3(s1.x / nn, s1.y / nn, s1.z / nn) : make_float3(0.f, 0.f, 1.f);
}

__global__ void puck_sums_brick_kernel(const Tri* __restrict__ tris, const int* __restrict__ brick_off, int nb,
                                       int64_t cap, float4* __restrict__ sums, unsigned* __restrict__ rth) {
  const int64_t nbr = (int64_t)nb * nb * nb;
  for (int64_t br = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; br < nbr;
       br += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = brick_off[br];
    const int64_t q1 = min((int64_t)brick_off[br + 1], cap);
    float3 cs = make_float3(0.f, 0.f, 0.f), ns = make_float3(0.f, 0.f, 0.f);
    for (int64_t q = q0; q < q1; ++q) {
      const Tri tr = tris[q];
      const float3 a = f3(tr.a), b = f3(tr.b), c = f3(tr.c);
      cs.x += a.x + b.x + c.x;
      cs.y += a.y + b.y + c.y;
      cs.z += a.z + b.z + c.z;
      const float3 cr = cross3(sub3(b, a), sub3(c, a));
      ns.x += cr.x;
      ns.y += cr.y;
      ns.z += cr.z;
    }
    sums[2 * br] = make_float4(cs.x, cs.y, cs.z, (float)(q1 > q0 ? q1 - q0 : 0));
    sums[2 * br + 1] = make_float4(ns.x, ns.y, ns.z, 0.f);
    rth[2 * br] = 0u;
    rth[2 * br + 1] = 0u;
  }
}

__global__ void puck_sums_up_kernel(float4* __restrict__ sums, unsigned* __restrict__ rth, int64_t a_child,
                                    int dchild, int64_t a_parent, int dparent) {
  const int64_t np = (int64_t)dparent * dparent * dparent;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < np;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t % dparent), y = (int)((t / dparent) % dparent), z = (int)(t / ((int64_t)dparent * dparent));
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < 8; ++q) {
      const int cx = 2 * x + (q & 1), cy = 2 * y + ((q >> 1) & 1), cz = 2 * z + (q >> 2);
      if (cx >= dchild || cy >= dchild || cz >= dchild) continue;
      const int64_t ci = a_child + ((int64_t)cz * dchild + cy) * dchild + cx;
      const float4 c0 = sums[2 * ci], c1 = sums[2 * ci + 1];
      s0 = make_float4(s0.x + c0.x, s0.y + c0.y, s0.z + c0.z, s0.w + c0.w);
      s1 = make_float4(s1.x + c1.x, s1.y + c1.y, s1.z + c1.z, 0.f);
    }
    sums[2 * (a_parent + t)] = s0;
    sums[2 * (a_parent + t) + 1] = s1;
    rth[2 * (a_parent + t)] = 0u;
    rth[2 * (a_parent + t) + 1] = 0u;
  }
}

__global__ void puck_rth_kernel(const Tri* __restrict__ tris, const int* __restrict__ leaf_off, int nb, int64_t cap,
                                PyrInfo pi, const int* __restrict__ live, const DevState* __restrict__ st,
                                const float4* __restrict__ sums, unsigned* __restrict__ rth) {
  const int dl = pi.dim[0];
  const int64_t nlive = st->nleaf_live;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the live leaves (list order keeps a warp's leaves together); warp-uniform
  // trip count: every lane reaches the warp-wide reductions
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nlive; base += stride) {
    const int64_t it = base + threadIdx.x;
    const bool in = it < nlive;
    const int64_t t = in ? live[it] : 0;
    const int lx = in ? (int)(t % dl) : 0, ly = in ? (int)((t / dl) % dl) : 0,
              lz = in ? (int)(t / ((int64_t)dl * dl)) : 0;
    int64_t q0 = 0, q1 = 0;
    if (in) {
      const int li = leaf_index(lx, ly, lz, nb);
      q0 = leaf_off[li];
      q1 = min((int64_t)leaf_off[li + 1], cap);
    }
#pragma unroll 1
    for (int l = 1; l < pi.nlev; ++l) {
      const int d = pi.dim[l];
      const int64_t node = ((int64_t)(lz >> l) * d + (ly >> l)) * d + (lx >> l);
      const int64_t a = pi.off[l] - pi.off[1] + node;
      float r = 0.f, th = 0.f;
      if (q1 > q0) {
        float3 c, ax;
        node_frame(sums[2 * a], sums[2 * a + 1], c, ax);
        for (int64_t q = q0; q < q1; ++q) {
          const Tri tr = tris[q];
          const float4 vv[3] = {tr.a, tr.b, tr.c};
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            const float3 dv = sub3(f3(vv[v]), c);
            const float zz = dot3(dv, ax);
            th = fmaxf(th, fabsf(zz));
            r = fmaxf(r, sqrtf(fmaxf(dot3(dv, dv) - zz * zz, 0.f)));
          }
        }
      }
      const long long key = (q1 > q0) ? (long long)a : -1ll;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const unsigned rm = __reduce_max_sync(peers, __float_as_uint(r));
      const unsigned tm = __reduce_max_sync(peers, __float_as_uint(th));
      if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
        atomicMax(&rth[2 * a], rm);
        atomicMax(&rth[2 * a + 1], tm);
      }
    }
  }
}

__global__ void puck_finalize_kernel(float4* __restrict__ pyr, const float4* __restrict__ sums,
                                     const unsigned* __restrict__ rth, int64_t naux, int64_t pyr_base) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < naux; a += (int64_t)gridDim.x * blockDim.x) {
    const float4 s0 = sums[2 * a], s1 = sums[2 * a + 1];
    const int64_t gi = pyr_base + a;
    if (!(s0.w > 0.f)) {
      pyr[2 * gi] = make_float4(0.f, 0.f, 0.f, -1.f);
      pyr[2 * gi + 1] = make_float4(0.f, 0.f, 1.f, 0.f);
      continue;
    }
    float3 c, ax;
    node_frame(s0, s1, c, ax);
    const float r = __uint_as_float(rth[2 * a]), th = __uint_as_float(rth[2 * a + 1]);
    const float pad = kPuckPad * (fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + r + th) + 1e-7f;
    pyr[2 * gi] = make_float4(c.x, c.y, c.z, r * (1.f + kPuckPad) + pad);
    pyr[2 * gi + 1] = make_float4(ax.x, ax.y, ax.z, th * (1.f + kPuckPad) + pad);
  }
}

// Child-occupancy masks of the internal nodes (levels >= 1): bit q set when
// child q (x + (q & 1), y + (q >> 1 & 1), z + (q >> 2), at twice the
// coordinates) exists and holds triangles.  The mask sits in the low 8 bits of
// the node's radius, rounded up first so that the stored radius never
// shrinks (the bound stays conservative; at most 2^-14 relative).
__global__ void puck_mask_kernel(float4* __restrict__ pyr, PyrInfo pi) {
  const int64_t total = pi.off[pi.nlev - 1] + 1 - pi.off[1];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = pi.off[1] + t;
    int l = 1;
    while (l + 1 < pi.nlev && gi >= pi.off[l + 1]) ++l;
    const float4 A = pyr[2 * gi];
    if (A.w < 0.f) continue;
    const int64_t r = gi - pi.off[l];
    const int d = pi.dim[l], dc = pi.dim[l - 1];
    const int x = (int)(r % d), y = (int)((r / d) % d), z = (int)(r / ((int64_t)d * d));
    unsigned mask = 0;
    for (int q = 0; q < 8; ++q) {
      const int cx = 2 * x + (q & 1), cy = 2 * y + ((q >> 1) & 1), cz = 2 * z + (q >> 2);
      if (cx >= dc || cy >= dc || cz >= dc) continue;
      const int64_t cg = pi.off[l - 1] + ((int64_t)cz * dc + cy) * dc + cx;
      if (pyr[2 * cg].w >= 0.f) mask |= 1u << q;
    }
    const unsigned up = (__float_as_uint(A.w) + 0xffu) & ~0xffu;
    pyr[2 * gi].w = __uint_as_float(up | mask);
  }
}

}  // namespace

namespace {

constexpr int kWarps = 4;          // warps per CTA
constexpr int kStack = 96;         // per-warp traversal stack

// Float32 rounding of one point-triangle distance, as a bound used to detect
// near-ties: relative to the distance, plus an absolute part for the rounding
// of the node and vertex coordinates (of magnitude up to the coordinate scale).
constexpr float kTieRel = 4e-7f;
constexpr float kTieAbs = 1.5e-7f;
constexpr int kCand = 4;           // smallest float32 distances kept per node
constexpr int kSdfCoarse = 2;      // stride of the coarsest (unseeded) search pass

struct TieSlots {
  int2* p[2];   // the two float-float iterate buffers; the one not current is free
};

// Squared distance from p to a triangle given by its search record (see
// write_search_record): the Voronoi region picks the closest point
// y = a + v ab + w ac (Ericson's case analysis, with the six dot products
// reduced to d1 = ab.ap and d2 = ac.ap through the stored Gram entries and
// the divisions replaced by the stored reciprocals), and the residual
// p - y = ap - v ab - w ac is formed relative to a, so its rounding scales
// with the distance and the edge length rather than with the coordinates.

__device__ __forceinline__ float tri_dist2_rec(const float3 p, const float4* __restrict__ rec, float& v, float& w,
                                               unsigned& vk) {
  const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
  const float3 ap = make_float3(p.x - r0.x, p.y - r0.y, p.z - r0.z);
  const float d1 = r1.x * ap.x + r1.y * ap.y + r1.z * ap.z;   // ab . ap
  const float d2 = r2.x * ap.x + r2.y * ap.y + r2.z * ap.z;   // ac . ap
  rec_weights(ap, d1, d2, r0, r1, r2, r3, v, w);
  vk = __float_as_uint(r1.w);
  const float rx = ap.x - v * r1.x - w * r2.x;
  const float ry = ap.y - v * r1.y - w * r2.y;
  const float rz = ap.z - v * r1.z - w * r2.z;
  return rx * rx + ry * ry + rz * rz;
}
__device__ __forceinline__ float tri_dist2_rec(const float3 p, const float4* __restrict__ rec) {
  float v, w;
  unsigned vk;
  return tri_dist2_rec(p, rec, v, w, vk);
}

// Key (32-bit hash; callers keep its top bits) of a node's closest feature on triangle t, from the weights
// (v, w) of its closest point y = a + v ab + w ac and the record's vertex
// hashes: a vertex (weights 0 / 1) by its hash, an edge (one weight 0, or
// v = 1 - w) by its two, a face by the triangle.  Triangles that share the
// closest vertex or edge give the same key.
__device__ __forceinline__ unsigned feature_key(float v, float w, unsigned vk, int t) {
  const unsigned ha = vk & 1023u, hb = (vk >> 10) & 1023u, hc = (vk >> 20) & 1023u;
  unsigned x;
  auto edge = [](unsigned p, unsigned q) { return (1u << 20) | (min(p, q) << 10) | max(p, q); };
  if (w == 0.f) {
    x = (v == 0.f) ? ha : (v == 1.f ? hb : edge(ha, hb));
  } else if (v == 0.f) {
    x = (w == 1.f) ? hc : edge(ha, hc);
  } else if (v == 1.f - w) {
    x = edge(hb, hc);
  } else {
    x = (2u << 20) ^ (unsigned)t;
  }
  return ((x * 0x9E3779B1u) ^ 0x7F4A7C15u) * 0x85EBCA6Bu;
}

// The same distance in float-float for the near-tie decisions.  Only ap and
// the residual need the extra precision: a region chosen wrongly near a
// region boundary, and rounding of the weights (v, w), change |p - y| only to
// second order (the residual is normal to the directions they move y in), so
// the region and the weights come from the float32 path; ap is formed in
// float-float from the float-float node position, v ab + w ac from exact
// products, and |p - y|^2 in float-float.
__device__ __forceinline__ Ff two_prod_ff(float a, float b) {
  const float p = __fmul_rn(a, b);
  return Ff(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ Ff tri_dist2_rec_ff(const Vec3<Ff> p, const float4* __restrict__ rec) {
  const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
  const Ff apx = p.x - Ff(r0.x), apy = p.y - Ff(r0.y), apz = p.z - Ff(r0.z);
  const float3 ap = make_float3(apx.hi, apy.hi, apz.hi);
  const float d1 = r1.x * ap.x + r1.y * ap.y + r1.z * ap.z;
  const float d2 = r2.x * ap.x + r2.y * ap.y + r2.z * ap.z;
  float v, w;
  rec_weights(ap, d1, d2, r0, r1, r2, r3, v, w);
  const Ff rx = apx - (two_prod_ff(v, r1.x) + two_prod_ff(w, r2.x));
  const Ff ry = apy - (two_prod_ff(v, r1.y) + two_prod_ff(w, r2.y));
  const Ff rz = apz - (two_prod_ff(v, r1.z) + two_prod_ff(w, r2.z));
  return rx * rx + ry * ry + rz * rz;
}

// The same on the ~48-bit vertices (float32 vertex + its low part, see
// mc_emit_kernel): a, ab and ac in float-float, so the distance is that of
// the refined surface to ~1e-14 relative and two candidates are ranked as
// the exact (FP64) mesh ranks them unless they tie to that level.  The region
// and the weights still come from the float32 record (second-order effect).
__device__ __forceinline__ Ff tri_dist2_ff_exact(const Vec3<Ff> p, const float4* __restrict__ rec, const Tri& hi,
                                                 const Tri& lo) {
  const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
  const Ff ax = Ff(hi.a.x) + Ff(lo.a.x), ay = Ff(hi.a.y) + Ff(lo.a.y), az = Ff(hi.a.z) + Ff(lo.a.z);
  const Ff abx = (Ff(hi.b.x) + Ff(lo.b.x)) - ax, aby = (Ff(hi.b.y) + Ff(lo.b.y)) - ay,
           abz = (Ff(hi.b.z) + Ff(lo.b.z)) - az;
  const Ff acx = (Ff(hi.c.x) + Ff(lo.c.x)) - ax, acy = (Ff(hi.c.y) + Ff(lo.c.y)) - ay,
           acz = (Ff(hi.c.z) + Ff(lo.c.z)) - az;
  const Ff apx = p.x - ax, apy = p.y - ay, apz = p.z - az;
  const float3 ap = make_float3(apx.hi, apy.hi, apz.hi);
  const float d1 = r1.x * ap.x + r1.y * ap.y + r1.z * ap.z;
  const float d2 = r2.x * ap.x + r2.y * ap.y + r2.z * ap.z;
  float v, w;
  rec_weights(ap, d1, d2, r0, r1, r2, r3, v, w);
  const Ff fv(v), fw(w);
  const Ff rx = apx - (fv * abx + fw * acx);
  const Ff ry = apy - (fv * aby + fw * acy);
  const Ff rz = apz - (fv * abz + fw * acz);
  return rx * rx + ry * ry + rz * rz;
}

// Octree entries on the traversal stack: level in bits 27..31, node
// coordinates (< 512 per axis) in bits 0..8 (x), 9..17 (y), 18..26 (z).  The
// search stacks this word with the node's pyramid index, so that a pop loads
// the node's puck at once instead of first looking up its level's offset and
// dimension.
__device__ __forceinline__ unsigned pack_node(int lev, int x, int y, int z) {
  return ((unsigned)lev << 27) | ((unsigned)z << 18) | ((unsigned)y << 9) | (unsigned)x;
}

// Warp-cooperative exact distance search: a warp owns a 4 x 4 x 2 patch of
// nodes and walks the octree once for all of them (a subtree is entered when
// its bound beats the current cut of at least one lane); in a leaf, the
// triangles of each MC cube whose own puck beats some lane's cut are tested
// by every lane against its own node with the same (broadcast) triangle.
//
// Exactness at near-ties: two triangles whose distances differ by less than
// the float32 rounding may be ranked either way, and the closest point (and
// with it the vertex gradient of Eqs. 35-36) differs between them.  Each lane
// keeps its kCand smallest float32 distances (four: triangles sharing the
// closest edge tie exactly, so candidates come in pairs) and prunes against
// the best plus a rounding margin; when the second lies within that margin
// the node is a near-tie: it is appended to tie_list, the ids of the
// candidates within the margin go to tie_a, tie_b and tie_cd at the same list
// position (-1 for none), and sdf_tie_kernel re-decides it in float-float.  Without TIES (no closest
// triangle is kept) the search keeps the float32 minimum alone, which is
// within the same rounding of the exact distance.
//
// Coarse to fine passes over nested lattices: pass `stride` S handles the
// nodes whose coordinates are all multiples of S but not all multiples of 2S
// (the coarsest pass, S = kSdfCoarse, takes all its lattice's nodes and
// starts from nothing).  A finer pass starts from the closest triangles of
// the up to 8 nodes of the 2S lattice around its node (seed_ids, written by
// every pass for its nodes): real triangle distances, so the cut is an upper
// bound from the start and the search mostly has to certify.
template <bool COUNT, bool TIES>
__global__ void __launch_bounds__(kWarps * 32, 10) sdf_kernel(const float* __restrict__ chi, SurfParams g,
                                                          DevState* __restrict__ st,
                                                          const float4* __restrict__ tris_s, int id_bits,
                                                          const int* __restrict__ leaf_off, int64_t cap,
                                                          const float4* __restrict__ pyr, PyrInfo pi,
                                                          float* __restrict__ phi, float* __restrict__ sdf_out,
                                                          int* __restrict__ ctri, int* __restrict__ tie_a,
                                                          int* __restrict__ tie_b, TieSlots tie_cd,
                                                          int* __restrict__ tie_list,
                                                          int* __restrict__ seed_ids, int stride,
                                                          const unsigned* __restrict__ leaf_cnt,
                                                          const float4* __restrict__ cell_pyr) {
  __shared__ uint2 s_node[kWarps][kStack];   // (packed level and coordinates, pyramid index)
  __shared__ int s_off[12];
  __shared__ int s_dim[12];
  if (threadIdx.x < 12) {
    s_off[threadIdx.x] = pi.off[threadIdx.x];
    s_dim[threadIdx.x] = pi.dim[threadIdx.x];
  }
  __syncthreads();
  const int n = g.res;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTA covers 8 x 8 x 2 nodes of this pass's lattice: warp w -> (4 (w & 1),
  // 4 (w >> 1)) in x, y
  const int S = stride;
  const bool seeded = S < kSdfCoarse;
  const int nl = (n + S - 1) / S;
  const int ntx = (nl + 7) / 8, nty = (nl + 7) / 8;
  const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
  const int i = S * (bx * 8 + 4 * (w & 1) + (lane & 3));
  const int j = S * (by * 8 + 4 * (w >> 1) + ((lane >> 2) & 3));
  const int k = S * (bz * 2 + (lane >> 4));
  const bool valid = (i < n) && (j < n) && (k < n) && (!seeded || ((i | j | k) & S));
  const int ic = min(i, n - 1), jc = min(j, n - 1), kc = min(k, n - 1);
  const float3 p = make_float3((float)(g.lo[0] + (ic + 0.5) * g.h), (float)(g.lo[1] + (jc + 0.5) * g.h),
                               (float)(g.lo[2] + (kc + 0.5) * g.h));
  constexpr int NC = TIES ? kCand : 1;
  float coord = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    coord = fmaxf(coord, (float)fmax(fabs(g.lo[a]), fabs(g.lo[a] + n * g.h)));
  const float mabs = kTieAbs * coord;
  float cd[NC];
  int ct[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    cd[q] = INFINITY;
    ct[q] = -1;
  }
  float cut = valid ? INFINITY : -INFINITY;   // a lane without a node never asks for a subtree
  // With id_bits > 0 (near-tie handles; triangle ids below 2^id_bits - 1,
  // id_bits <= 24) each list entry carries the top 32 - id_bits bits of its
  // closest feature's key (feature_key) above the id, and the list holds one
  // entry per closest feature:
  // triangles sharing the closest vertex (often six of them) or edge tie
  // exactly and would otherwise fill the list and push out a distinct surface
  // point at the same distance (a node on the medial axis), which the tie
  // pass must see.  Entries merge when their keys match; both lie within the
  // rounding margin of the best, so a key collision can at most leave a tie
  // to the float32 ranking.
  const bool keyed = TIES && id_bits > 0;
  const int idmask = keyed ? (int)((1u << id_bits) - 1u) : -1;
  auto margin2 = [&](float x) {
    const float r = sqrtf(x) * (1.f + kTieRel) + mabs;
    return r * r;
  };
  // candidate list insertion (sorted, duplicates of a listed triangle ignored)
  auto offer = [&](float d2, int t, float v, float w, unsigned vk) {
    if (!(d2 < cut && d2 < cd[NC - 1])) return;
    int e = t;
    int at = NC - 1;
    if (keyed) {
      const unsigned key = feature_key(v, w, vk, t) >> id_bits;
      e = t | (int)(key << id_bits);
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        if ((ct[q] & idmask) == t) return;
        if (ct[q] != -1 && ((unsigned)ct[q] >> id_bits) == key) {
          if (!(d2 < cd[q])) return;      // the listed entry of this feature stays
          at = q;                         // replaced in place, then moved up
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < NC; ++q)
        if (ct[q] == t) return;
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {   // static indices: the list stays in registers
      if (q == at) {
        cd[q] = d2;
        ct[q] = e;
      }
    }
#pragma unroll
    for (int q = NC - 1; q > 0; --q) {
      if (q <= at && cd[q] < cd[q - 1]) {
        const float tf = cd[q];
        cd[q] = cd[q - 1];
        cd[q - 1] = tf;
        const int ti = ct[q];
        ct[q] = ct[q - 1];
        ct[q - 1] = ti;
      }
    }
    if (TIES) {
      cut = margin2(cd[0]);
    } else {
      cut = cd[0];
    }
  };
  if (seeded && valid) {
    // seeds: the closest triangles of the 2S-lattice nodes around this node
    const int S2 = 2 * S;
    const int i0 = i & ~(S2 - 1), j0 = j & ~(S2 - 1), k0 = k & ~(S2 - 1);
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const int ii = i0 + S2 * (q & 1), jj = j0 + S2 * ((q >> 1) & 1), kk = k0 + S2 * (q >> 2);
      if (ii >= n || jj >= n || kk >= n) continue;
      const int t = seed_ids[lin3(ii, jj, kk, n)];
      if (t >= 0) {
        float v, w;
        unsigned vk;
        const float d2 = tri_dist2_rec(p, tris_s + kTriRec * (int64_t)t, v, w, vk);
        offer(d2, t, v, w, vk);
      }
    }
  }
  uint2* stk = s_node[w];
  int sp = 0;
  const int top = pi.nlev - 1;
  const int nb = (s_dim[0] + 1) / 2;
  if (lane == 0) stk[0] = make_uint2(pack_node(top, 0, 0, 0), (unsigned)s_off[top]);
  sp = 1;
  unsigned long long c_nodes = 0, c_leaves = 0, c_tests = 0;
  // the warp's nodes' bounding box: centre and half-diagonal, widened so that
  // float rounding keeps the box bound below every lane's exact bound
  float bc[3], br;
  {
    const float pv[3] = {p.x, p.y, p.z};
    float r2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float lo = pv[a], hi = pv[a];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      bc[a] = 0.5f * (lo + hi);
      const float e = 0.5f * (hi - lo);
      r2 += e * e;
    }
    br = sqrtf(r2) * (1.f + 1e-5f) + 1e-7f * coord;
  }
  const float3 pb = make_float3(bc[0], bc[1], bc[2]);
  __syncwarp();
  while (sp > 0) {
    --sp;
    const uint2 en = stk[sp];
    __syncwarp();
    const unsigned e = en.x;
    const int gi = (int)en.y;
    const int lev = (int)(e >> 27);
    const int x = (int)(e & 511u), y = (int)((e >> 9) & 511u), z = (int)((e >> 18) & 511u);
    const float4 An = pyr[2 * gi];
    const float lb = puck_dist2(p, An, pyr[2 * gi + 1]);
    if (!__any_sync(0xffffffffu, lb < cut)) continue;
    if (COUNT) ++c_nodes;
    if (lev == 0) {
      const int li = leaf_index(x, y, z, nb);
      const int s1 = (int)min((int64_t)leaf_off[li + 1], cap);
      if (COUNT) ++c_leaves;
      // the leaf's cubes in order; a cube's triangles are tested when its
      // own puck beats the cut of at least one lane
      unsigned cn = leaf_cnt[li];
      int q0 = leaf_off[li];
#pragma unroll 1
      for (; cn != 0u; cn >>= 4) {
        const int q1 = min(q0 + (int)(cn & 15u), s1);
        if (q0 < q1 &&
            __any_sync(0xffffffffu, puck_dist2(p, cell_pyr[2 * q0], cell_pyr[2 * q0 + 1]) < cut)) {
          if (COUNT) c_tests += 32ull * (unsigned long long)(q1 - q0);
          for (int t = q0; t < q1; ++t) {
            float v, w;
            unsigned vk;
            const float d2 = tri_dist2_rec(p, tris_s + kTriRec * t, v, w, vk);
            offer(d2, t, v, w, vk);
          }
        }
        q0 += (int)(cn & 15u);
      }
      continue;
    }
    const int dc = s_dim[lev - 1];
    const int cbase = s_off[lev - 1];
    // children, one per lane (lanes 0-7): kept when their bound from the
    // warp's box (the puck's distance to the box centre less the box's
    // half-diagonal, a lower bound for every node in it) beats the largest
    // lane cut; pushed far-to-near by that bound in the unseeded pass, in
    // child order in the seeded ones (their cuts start near their final
    // values, so the order saves little and the ranking costs 8 shuffles).
    // Each lane's own bound is checked when a child is popped, so a child is
    // bounded per lane once.
    const unsigned cmask = __float_as_uint(An.w) & 0xffu;
    const float maxcut = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(cut, 0.f))));
    bool keep = false;
    float key = INFINITY;
    uint2 ent = make_uint2(0u, 0u);
    if (lane < 8 && ((cmask >> lane) & 1u)) {
      const int cx = 2 * x + (lane & 1), cy = 2 * y + ((lane >> 1) & 1), cz = 2 * z + (lane >> 2);
      const int cg = cbase + (cz * dc + cy) * dc + cx;
      const float dcen = sqrtf(puck_dist2(pb, pyr[2 * cg], pyr[2 * cg + 1])) * (1.f - 2e-6f) - br;
      key = dcen > 0.f ? dcen * dcen : 0.f;
      keep = key < maxcut;
      ent = make_uint2(pack_node(lev - 1, cx, cy, cz), (unsigned)cg);
    }
    const unsigned kept = __ballot_sync(0xffffffffu, keep);
    const int nc = __popc(kept);
    int rank = 0;   // kept children nearer than this one (ties by lane)
    if (seeded) {
      rank = nc - 1 - __popc(kept & ((1u << lane) - 1u));
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float kq = __shfl_sync(0xffffffffu, key, q);
        if (((kept >> q) & 1u) && (kq < key || (kq == key && q < lane))) ++rank;
      }
    }
    const int slot = sp + nc - 1 - rank;
    if (keep && slot < kStack) stk[slot] = ent;
    sp = min(sp + nc, kStack);
    __syncwarp();
  }
  const bool tie = TIES && valid && ct[NC > 1 ? 1 : 0] != -1 && cd[NC > 1 ? 1 : 0] <= cut;
  if (COUNT) {
    const unsigned long long nt = (unsigned long long)__popc(__ballot_sync(0xffffffffu, tie));
    if (lane == 0) {
      atomicAdd(&st->sdf_cnt[0], c_nodes);
      atomicAdd(&st->sdf_cnt[1], c_leaves);
      atomicAdd(&st->sdf_cnt[2], c_tests);
      atomicAdd(&st->sdf_cnt[3], nt);
    }
  }
  const int64_t o = lin3(i, j, k, n);
  int tie_at = 0;
  if (TIES) {
    // near-tie nodes go to a compact list (one atomic per warp), so that the
    // tie pass runs full warps over them alone; their candidates are stored
    // at the same list position (read coalesced by the tie pass)
    const unsigned m = __ballot_sync(0xffffffffu, tie);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(&st->ntie, (unsigned)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      tie_at = (int)(base + __popc(m & ((1u << lane) - 1u)));
      if (tie) tie_list[tie_at] = (int)o;
    }
  }
  if (!valid) return;
  const float val = sqrtf(cd[0]);
  const int bt = ct[0] == -1 ? -1 : (ct[0] & idmask);
  const float sgn = (chi[o] >= st->c_up) ? 1.f : -1.f;
  phi[o] = sgn * val;
  if (sdf_out) sdf_out[o] = sgn * val;
  if (ctri) ctri[o] = bt;
  if (S > 1) seed_ids[o] = bt;
  if (TIES && tie) {
    tie_a[tie_at] = bt;
    tie_b[tie_at] = ct[NC > 1 ? 1 : 0] & idmask;
    const int c2 = ct[NC > 2 ? 2 : 0], c3 = ct[NC > 3 ? 3 : 0];
    tie_cd.p[st->fwd.xidx ^ 1][tie_at] = make_int2(cd[NC > 2 ? 2 : 0] <= cut && c2 != -1 ? (c2 & idmask) : -1,
                                                   cd[NC > 3 ? 3 : 0] <= cut && c3 != -1 ? (c3 & idmask) : -1);
  }
}

// Float-float decision between the float32 near-tie candidates of a node:
// distances (tri_dist2_ff_exact on the ~48-bit vertices when their low parts
// exist, else tri_dist2_rec_ff on the float32 ones) from the node position
// rounded once from double, the smaller wins; equal distances (a shared edge or vertex: the
// same closest point) take the smaller triangle index.  The node coordinates come from per-axis
// float-float tables built once per block, and chi >= c (c double) is tested
// as chi >= the smallest float not below c, so no node needs FP64.

__global__ void sdf_tie_kernel(const float* __restrict__ chi, SurfParams g, const DevState* __restrict__ st,
                               const float4* __restrict__ tris_s, const Tri* __restrict__ tris,
                               const Tri* __restrict__ tris_lo, const int* __restrict__ tie_a,
                               const int* __restrict__ tie_b, TieSlots tie_cd, const int* __restrict__ tie_list,
                               float* __restrict__ phi, float* __restrict__ sdf_out, int* __restrict__ ctri) {
  __shared__ float2 s_ax[3][kMaxRes];
  const int n = g.res;
  for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
    const int a = t / n, i = t % n;
    const double v = g.lo[a] + (i + 0.5) * g.h;
    const float hi = (float)v;
    s_ax[a][i] = make_float2(hi, (float)(v - (double)hi));
  }
  __syncthreads();
  const float cf = st->c_up;
  const unsigned un = (unsigned)n;
  const unsigned count = st->ntie;
  const int xi = st->fwd.xidx ^ 1;
  for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < count; it += gridDim.x * blockDim.x) {
    const unsigned o = (unsigned)tie_list[it];
    const int t1 = tie_b[it];
    const int t0 = tie_a[it];
    const int2 t23 = tie_cd.p[xi][it];
    const unsigned row = o / un;
    const int i = (int)(o - row * un), j = (int)(row % un), k = (int)(row / un);
    const float2 px = s_ax[0][i], py = s_ax[1][j], pz = s_ax[2][k];
    const Vec3<Ff> pf = {Ff(px.x, px.y), Ff(py.x, py.y), Ff(pz.x, pz.y)};
    Ff bd(INFINITY);
    int bi = -1;
    const int cand[kCand] = {t0, t1, t23.x, t23.y};
    // one copy of the float-float distance in the loop: unrolled, the four
    // copies overflow the instruction cache
#pragma unroll 1
    for (int q = 0; q < kCand; ++q) {
      if (cand[q] < 0) continue;
      const Ff d2 = tris_lo ? tri_dist2_ff_exact(pf, tris_s + kTriRec * (int64_t)cand[q], tris[cand[q]],
                                                 tris_lo[cand[q]])
                            : tri_dist2_rec_ff(pf, tris_s + kTriRec * (int64_t)cand[q]);
      if (bi < 0 || d2 < bd || (!(bd < d2) && cand[q] < bi)) {
        bd = d2;
        bi = cand[q];
      }
    }
    const float sgn = (chi[o] >= cf) ? 1.f : -1.f;
    const float val = sgn * sqrtf(__fadd_rn(bd.hi, bd.lo));
    phi[o] = val;
    if (sdf_out) sdf_out[o] = val;
    ctri[o] = bi;
  }
}

// n = grad phi / |grad phi|: central differences inside, second-order one-sided
// on the first and last node of each axis; 0 where |grad| is 0 or not finite.
// One thread per (x, y) column marches kNrmZ planes in z, keeping the
// column's previous, current and next phi in registers; x and y neighbours
// come through L1 from the warp's own row and the block's neighbouring rows.
// No index division, coalesced loads and stores of every plane.
constexpr int kNrmZ = 16;
__global__ void __launch_bounds__(256) normals_kernel(const float* __restrict__ phi, int n, double h,
                                                      float* __restrict__ nrm) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  const int k0 = blockIdx.z * kNrmZ;
  if (i >= n || j >= n || k0 >= n) return;
  const int64_t nn = (int64_t)n * n, N = nn * n;
  const float inv2h = (float)(0.5 / h);
  const int k1 = min(k0 + kNrmZ, n);
  int64_t t = (int64_t)k0 * nn + (int64_t)j * n + i;
  float zm = k0 > 0 ? phi[t - nn] : 0.f;
  float zc = phi[t];
  for (int k = k0; k < k1; ++k, t += nn) {
    const float zp = k + 1 < n ? phi[t + nn] : 0.f;
    float gr[3];
    if (i == 0)
      gr[0] = -3.f * zc + 4.f * phi[t + 1] - phi[t + 2];
    else if (i == n - 1)
      gr[0] = 3.f * zc - 4.f * phi[t - 1] + phi[t - 2];
    else
      gr[0] = phi[t + 1] - phi[t - 1];
    if (j == 0)
      gr[1] = -3.f * zc + 4.f * phi[t + n] - phi[t + 2 * n];
    else if (j == n - 1)
      gr[1] = 3.f * zc - 4.f * phi[t - n] + phi[t - 2 * n];
    else
      gr[1] = phi[t + n] - phi[t - n];
    if (k == 0)
      gr[2] = -3.f * zc + 4.f * zp - phi[t + 2 * nn];
    else if (k == n - 1)
      gr[2] = 3.f * zc - 4.f * zm + phi[t - 2 * nn];
    else
      gr[2] = zp - zm;
#pragma unroll
    for (int a = 0; a < 3; ++a) gr[a] *= inv2h;
    const float m2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    const bool ok = isfinite(m2) && m2 > 0.f;
    const float inv = ok ? rsqrtf(m2) : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) nrm[a * N + t] = ok ? gr[a] * inv : 0.f;
    zm = zc;
    zc = zp;
  }
}

// ---- exact signed distance at arbitrary query points (Sec. 2.4, Eqs. 29-34,
// evaluated off the grid).  Two kernels: the distance search over queries
// sorted by cell (a warp of 32 neighbouring queries walks the octree as the
// node search does), then the sign, one thread per query.

// Distance search.  The cut starts from an upper bound: the nearest node's
// |phi| plus the node's distance to q (triangle inequality), widened for the
// float rounding of both; with the nodes' closest triangles kept (SEEDS),
// those of the 8 nodes around q are offered first.  Writes the unsigned distance and the unit
// direction (q - y) / |q - y| to the closest surface point y (zero when q is
// on the surface, infinite distance when the mesh is empty).
template <bool SEEDS>
__global__ void __launch_bounds__(kWarps * 32, 8) sdf_query_kernel(const float* __restrict__ phi, SurfParams g,
                                                                const Tri* __restrict__ tris,
                                                                const float4* __restrict__ tris_s,
                                                                const int* __restrict__ leaf_off, int64_t cap,
                                                                const float4* __restrict__ pyr, PyrInfo pi,
                                                                const float4* __restrict__ sorted,
                                                                const int* __restrict__ total,
                                                                const int* __restrict__ ctri,
                                                                float* __restrict__ dist_out,
                                                                float* __restrict__ dir_out,
                                                                int* __restrict__ tri_out) {
  __shared__ uint2 s_node[kWarps][kStack];   // (packed level and coordinates, pyramid index)
  __shared__ int s_off[12];
  __shared__ int s_dim[12];
  if (threadIdx.x < 12) {
    s_off[threadIdx.x] = pi.off[threadIdx.x];
    s_dim[threadIdx.x] = pi.dim[threadIdx.x];
  }
  __syncthreads();
  const int m = *total;
  const int n = g.res;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float coord = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    coord = fmaxf(coord, (float)fmax(fabs(g.lo[a]), fabs(g.lo[a] + n * g.h)));
  const int top = pi.nlev - 1;
  const int nb = (s_dim[0] + 1) / 2;
  uint2* stk = s_node[w];
  const int nwarps = gridDim.x * kWarps;
  for (int base = (blockIdx.x * kWarps + w) * 32; base < m; base += nwarps * 32) {
    const int k = base + lane;
    const bool valid = k < m;
    const float4 e = sorted[valid ? k : base];
    const float3 p = make_float3(e.x, e.y, e.z);
    // nearest node and the bound |phi(node)| + |q - node|
    int ni[3];
    const float pq[3] = {e.x, e.y, e.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double f = ((double)pq[a] - g.lo[a]) / g.h - 0.5;
      ni[a] = (int)fmin(fmax(rint(f), 0.0), (double)(n - 1));
    }
    const int64_t o = lin3(ni[0], ni[1], ni[2], n);
    const float3 nd = make_float3((float)(g.lo[0] + (ni[0] + 0.5) * g.h), (float)(g.lo[1] + (ni[1] + 0.5) * g.h),
                                  (float)(g.lo[2] + (ni[2] + 0.5) * g.h));
    const float dn = sqrtf((p.x - nd.x) * (p.x - nd.x) + (p.y - nd.y) * (p.y - nd.y) + (p.z - nd.z) * (p.z - nd.z));
    const float bnd = (fabsf(phi[o]) + dn) * (1.f + 1e-5f) + 1e-6f * coord;
    float cut = valid ? bnd * bnd : -INFINITY;
    float cd = INFINITY;
    int ct = -1;
    auto offer = [&](float d2, int t) {
      if (d2 < cut && d2 < cd) {
        cd = d2;
        ct = t;
        cut = d2;
      }
    };
    if (SEEDS && valid) {
      // the closest triangles of the 8 nodes around q
      int c0[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double f = ((double)pq[a] - g.lo[a]) / g.h - 0.5;
        c0[a] = (int)fmin(fmax(floor(f), 0.0), (double)(n - 2));
      }
#pragma unroll 1
      for (int qn = 0; qn < 8; ++qn) {
        const int t = ctri[lin3(c0[0] + (qn & 1), c0[1] + ((qn >> 1) & 1), c0[2] + (qn >> 2), n)];
        if (t >= 0) offer(tri_dist2_rec(p, tris_s + kTriRec * (int64_t)t), t);
      }
    }
    int sp = 1;
    if (lane == 0) stk[0] = make_uint2(pack_node(top, 0, 0, 0), (unsigned)s_off[top]);
    __syncwarp();
    while (sp > 0) {
      --sp;
      const uint2 ew = stk[sp];
      __syncwarp();
      const unsigned en = ew.x;
      const int gi = (int)ew.y;
      const int lev = (int)(en >> 27);
      const int x = (int)(en & 511u), y = (int)((en >> 9) & 511u), z = (int)((en >> 18) & 511u);
      const float4 An = pyr[2 * gi];
      const float lb = puck_dist2(p, An, pyr[2 * gi + 1]);
      if (!__any_sync(0xffffffffu, lb < cut)) continue;
      if (lev == 0) {
        const int li = leaf_index(x, y, z, nb);
        const int64_t s0 = leaf_off[li];
        const int64_t s1 = min((int64_t)leaf_off[li + 1], cap);
        for (int64_t t = s0; t < s1; ++t) offer(tri_dist2_rec(p, tris_s + kTriRec * t), (int)t);
        continue;
      }
      const int dc = s_dim[lev - 1];
      const int cbase = s_off[lev - 1];
      float key[8];
      uint2 ent[8];
      int nc = 0;
      const unsigned cmask = __float_as_uint(An.w) & 0xffu;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!((cmask >> q) & 1u)) continue;
        const int cx = 2 * x + (q & 1), cy = 2 * y + ((q >> 1) & 1), cz = 2 * z + (q >> 2);
        const int cg = cbase + (cz * dc + cy) * dc + cx;
        const float d = puck_dist2(p, pyr[2 * cg], pyr[2 * cg + 1]);
        if (!__any_sync(0xffffffffu, d < cut)) continue;
        const float dm = __shfl_sync(0xffffffffu, d, 0);
        int q2 = nc;
        while (q2 > 0 && key[q2 - 1] < dm) {
          key[q2] = key[q2 - 1];
          ent[q2] = ent[q2 - 1];
          --q2;
        }
        key[q2] = dm;
        ent[q2] = make_uint2(pack_node(lev - 1, cx, cy, cz), (unsigned)cg);
        ++nc;
      }
      if (lane == 0)
        for (int q = 0; q < nc && sp + q < kStack; ++q) stk[sp + q] = ent[q];
      sp = min(sp + nc, kStack);
      __syncwarp();
    }
    if (!valid) continue;
    const int idx = __float_as_int(e.w);
    float3 dir = make_float3(0.f, 0.f, 0.f);
    if (ct >= 0 && cd > 0.f) {
      // residual q - y of the closest point y, as in the distance itself
      const float4* rec = tris_s + kTriRec * (int64_t)ct;
      const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
      const float3 ap = make_float3(p.x - r0.x, p.y - r0.y, p.z - r0.z);
      const float d1 = r1.x * ap.x + r1.y * ap.y + r1.z * ap.z;
      const float d2 = r2.x * ap.x + r2.y * ap.y + r2.z * ap.z;
      float v, wt;
      rec_weights(ap, d1, d2, r0, r1, r2, r3, v, wt);
      const float3 r = make_float3(ap.x - v * r1.x - wt * r2.x, ap.y - v * r1.y - wt * r2.y,
                                   ap.z - v * r1.z - wt * r2.z);
      const float len = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
      if (len > 0.f) dir = make_float3(r.x / len, r.y / len, r.z / len);
      if (!(r0.w * r2.w * r3.w < kSliverKappa)) {
        // a sliver: the closest point's direction in FP64
        const Tri tr = tris[ct];
        const double pd[3] = {p.x, p.y, p.z}, ad[3] = {tr.a.x, tr.a.y, tr.a.z}, bd[3] = {tr.b.x, tr.b.y, tr.b.z},
                     cdv[3] = {tr.c.x, tr.c.y, tr.c.z};
        double bw64[3], dir64[3];
        closest_point_fp64(pd, ad, bd, cdv, bw64, dir64);
        dir = make_float3((float)dir64[0], (float)dir64[1], (float)dir64[2]);
      }
    }
    dist_out[idx] = ct >= 0 ? sqrtf(cd) : INFINITY;
    if (tri_out) tri_out[idx] = ct;
    if (dir_out) {
      dir_out[3 * (int64_t)idx] = dir.x;
      dir_out[3 * (int64_t)idx + 1] = dir.y;
      dir_out[3 * (int64_t)idx + 2] = dir.z;
    }
  }
}

__device__ __forceinline__ float orient3(float3 a, float3 b, float3 c, float3 d) {
  // (a - d) . ((b - d) x (c - d))
  const float3 ad = make_float3(a.x - d.x, a.y - d.y, a.z - d.z);
  const float3 bd = make_float3(b.x - d.x, b.y - d.y, b.z - d.z);
  const float3 cd = make_float3(c.x - d.x, c.y - d.y, c.z - d.z);
  return ad.x * (bd.y * cd.z - bd.z * cd.y) + ad.y * (bd.z * cd.x - bd.x * cd.z) + ad.z * (bd.x * cd.y - bd.y * cd.x);
}

// Squared distance from p to triangle (a, b, c): the closest point by Voronoi
// regions (Ericson, Real-Time Collision Detection, 5.1.5), in float.
__device__ float pt_tri_dist2(float3 p, float3 a, float3 b, float3 c) {
  const float3 ab = sub3(b, a), ac = sub3(c, a), ap = sub3(p, a);
  const float d1 = dot3(ab, ap), d2 = dot3(ac, ap);
  float3 y;
  if (d1 <= 0.f && d2 <= 0.f) {
    y = a;
  } else {
    const float3 bp = sub3(p, b);
    const float d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    const float3 cp = sub3(p, c);
    const float d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    const float vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
    if (d3 >= 0.f && d4 <= d3) {
      y = b;
    } else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
      const float t = d1 / (d1 - d3);
      y = make_float3(a.x + t * ab.x, a.y + t * ab.y, a.z + t * ab.z);
    } else if (d6 >= 0.f && d5 <= d6) {
      y = c;
    } else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
      const float t = d2 / (d2 - d6);
      y = make_float3(a.x + t * ac.x, a.y + t * ac.y, a.z + t * ac.z);
    } else if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
      const float t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
      y = make_float3(b.x + t * (c.x - b.x), b.y + t * (c.y - b.y), b.z + t * (c.z - b.z));
    } else {
      const float den = va + vb + vc;
      const float v = den != 0.f ? vb / den : 0.f, ww = den != 0.f ? vc / den : 0.f;
      y = make_float3(a.x + v * ab.x + ww * ac.x, a.y + v * ab.y + ww * ac.y, a.z + v * ab.z + ww * ac.z);
    }
  }
  const float3 r = sub3(p, y);
  return dot3(r, r);
}

// Sign of every query by a parity test local to the cube that holds it (the
// query clamped into the node hull, where no triangle lies between it and its
// clamp): the segment from q to a corner v of the cube stays in the cube, so
// only that cube's marching-cubes triangles, regenerated from chi exactly as
// mc_emit_kernel writes them, can cross it; v's class is known (chi < c
// inside), and an odd number of crossings gives q the other class.  v is the
// corner farthest from the cube's triangles, so no triangle passes within
// rounding of it, among the corners off every cube face that q lies on (so
// the open segment avoids the faces, where triangles of the neighbouring cubes
// meet this cube's); q exactly at a corner takes that node's class.  A crossing needs q and v strictly on opposite sides of the
// triangle's plane and the line qv inside the triangle: the three orientations
// of the line against the triangle's edges agree in sign.  Each edge's
// orientation is evaluated once, in the order of its endpoints' global edge
// ids, and negated for the triangle that runs it the other way, so a line
// through an edge shared by two triangles counts for exactly one of them.  A
// float orientation can be wrong only when q lies within rounding of a
// triangle, where |phi| is of rounding size.  Non-finite queries get NaN and a
// zero gradient.
__global__ void query_sign_kernel(const float* __restrict__ q, int64_t m, const float* __restrict__ chi,
                                  ChiFF chiff, SurfParams g, const DevState* __restrict__ st,
                                  float* __restrict__ sdf_q, float* __restrict__ nrm_q) {
  const int n = g.res;
  const double c = st->c;
  const float c_up = st->c_up;
  const float2* __restrict__ xff = chiff.p[0] ? chiff.p[st->fwd.xidx] : nullptr;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const float x0 = q[3 * t], x1 = q[3 * t + 1], x2 = q[3 * t + 2];
    if (!(isfinite(x0) && isfinite(x1) && isfinite(x2))) {
      sdf_q[t] = __int_as_float(0x7fc00000);
      if (nrm_q) nrm_q[3 * t] = nrm_q[3 * t + 1] = nrm_q[3 * t + 2] = 0.f;
      continue;
    }
    const float xs[3] = {x0, x1, x2};
    float qc[3];
    int cc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double lo = g.lo[a] + 0.5 * g.h, hi = g.lo[a] + (n - 0.5) * g.h;
      const double v = fmin(fmax((double)xs[a], lo), hi);
      qc[a] = (float)v;
      cc[a] = min((int)floor((v - g.lo[a]) / g.h - 0.5), n - 2);
      cc[a] = max(cc[a], 0);
    }
    const int code = cube_code(chi, cc[0], cc[1], cc[2], n, c_up);
    // faces of the cube that q lies on: the segment's corner must be on the
    // opposite face, so that the open segment runs inside the cube (where only
    // this cube's triangles are); at a corner q takes that node's class
    int need_hi = 0, need_lo = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float flo = (float)(g.lo[a] + (cc[a] + 0.5) * g.h), fhi = (float)(g.lo[a] + (cc[a] + 1.5) * g.h);
      if (qc[a] == flo) need_hi |= 1 << a;
      if (qc[a] == fhi) need_lo |= 1 << a;
    }
    bool inside;
    if ((need_hi | need_lo) == 7) {
      const int corner = (need_lo & 1) | (((need_lo >> 1) & 1) << 1) | (((need_lo >> 2) & 1) << 2);
      inside = ((code >> corner) & 1) != 0;
    } else if (code == 0 || code == 255) {
      inside = code == 255;
    } else {
      // the cube's triangles
      float3 vt[kMaxTriPerCube][3];
      int gid[kMaxTriPerCube][3];
      const int ntri = c_mc_count[code];
      for (int tr = 0; tr < ntri; ++tr)
        for (int v = 0; v < 3; ++v) {
          const int ed = c_mc_tris[code][tr][v];
          int ox, oy, oz, ax;
          edge_lower_offset(ed, ox, oy, oz, ax);
          const int pi = cc[0] + ox, pj = cc[1] + oy, pk = cc[2] + oz;
          const int64_t pl = lin3(pi, pj, pk, n);
          const int64_t stride = (ax == 0) ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
          double c1, c2;
          if (xff) {
            const float2 f1 = xff[pl], f2 = xff[pl + stride];
            c1 = (double)f1.x + (double)f1.y;
            c2 = (double)f2.x + (double)f2.y;
          } else {
            c1 = (double)chi[pl];
            c2 = (double)chi[pl + stride];
          }
          const double eta = (c - c1) / (c2 - c1);
          double pos[3] = {g.lo[0] + (pi + 0.5) * g.h, g.lo[1] + (pj + 0.5) * g.h, g.lo[2] + (pk + 0.5) * g.h};
          pos[ax] += eta * g.h;
          vt[tr][v] = make_float3((float)pos[0], (float)pos[1], (float)pos[2]);
          gid[tr][v] = (int)(3 * pl + ax);
        }
      // the corner farthest from the triangles
      int best_c = 0;
      float best_d = -1.f;
      float3 vpos = make_float3(0.f, 0.f, 0.f);
      for (int qn = 0; qn < 8; ++qn) {
        if ((qn & need_hi) != need_hi || (qn & need_lo) != 0) continue;
        const float3 cp = make_float3((float)(g.lo[0] + (cc[0] + (qn & 1) + 0.5) * g.h),
                                      (float)(g.lo[1] + (cc[1] + ((qn >> 1) & 1) + 0.5) * g.h),
                                      (float)(g.lo[2] + (cc[2] + (qn >> 2) + 0.5) * g.h));
        float dmin = INFINITY;
        for (int tr = 0; tr < ntri; ++tr) dmin = fminf(dmin, pt_tri_dist2(cp, vt[tr][0], vt[tr][1], vt[tr][2]));
        if (dmin > best_d) {
          best_d = dmin;
          best_c = qn;
          vpos = cp;
        }
      }
      const float3 qp = make_float3(qc[0], qc[1], qc[2]);
      int cross = 0;
      for (int tr = 0; tr < ntri; ++tr) {
        const float sq = orient3(vt[tr][0], vt[tr][1], vt[tr][2], qp);
        const float sv = orient3(vt[tr][0], vt[tr][1], vt[tr][2], vpos);
        if (!((sq > 0.f && sv < 0.f) || (sq < 0.f && sv > 0.f))) continue;
        int sg[3];
        for (int ei = 0; ei < 3; ++ei) {
          const int a = ei, b = (ei + 1) % 3;
          const bool fwd = gid[tr][a] < gid[tr][b];
          const float3 A = fwd ? vt[tr][a] : vt[tr][b], B = fwd ? vt[tr][b] : vt[tr][a];
          const int sgn = orient3(qp, vpos, A, B) >= 0.f ? 1 : -1;
          sg[ei] = fwd ? sgn : -sgn;
        }
        cross += (sg[0] == sg[1] && sg[1] == sg[2]) ? 1 : 0;
      }
      inside = (((code >> best_c) & 1) != 0) != ((cross & 1) != 0);
    }
    if (inside) {
      sdf_q[t] = -sdf_q[t];
      if (nrm_q) {
        nrm_q[3 * t] = -nrm_q[3 * t];
        nrm_q[3 * t + 1] = -nrm_q[3 * t + 1];
        nrm_q[3 * t + 2] = -nrm_q[3 * t + 2];
      }
    }
  }
}

PyrInfo pyramid_info(int nl) {
  PyrInfo pi;
  int d = nl;
  long long off = 0;
  pi.nlev = 0;
  while (true) {
    pi.dim[pi.nlev] = d;
    pi.off[pi.nlev] = off;
    off += (long long)d * d * d;
    ++pi.nlev;
    if (d == 1) break;
    d = (d + 1) / 2;
  }
  return pi;
}

}  // namespace

// nb = bricks per axis; the octree's leaves are the 2 nb sub-bricks per axis
size_t pyramid_nodes(int nb) {
  PyrInfo pi = pyramid_info(2 * nb);
  return (size_t)(pi.off[pi.nlev - 1] + 1);
}

size_t pyramid_aux_nodes(int nb) {
  PyrInfo pi = pyramid_info(2 * nb);
  return (size_t)(pi.off[pi.nlev - 1] + 1 - pi.off[1]);
}

int launch_isovalue(wgeo_handle* h, const float* points, int64_t n, int res, cudaStream_t s) {
  SurfParams g;
  for (int a = 0; a < 3; ++a) g.lo[a] = h->lo[a];
  g.h = h->h;
  g.res = res;
  g.nb = div_up(res - 1, kBrick);
  const int nbk = grid_blocks(n, 256, kPartials);
  if (n > 0) {
    isovalue_kernel<<<nbk, 256, 0, s>>>(points, n, h->pcell, h->chi32, g, h->partials);
    WGEO_LAUNCH_CHECK();
  } else {
    WGEO_CUDA_TRY(cudaMemsetAsync(h->partials, 0, 2 * sizeof(double), s));
  }
  isovalue_finalize_kernel<<<1, 1024, 0, s>>>(h->partials, n > 0 ? nbk : 1, h->dstate);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

int launch_mc_sdf_normals(wgeo_handle* h, int res, float* sdf_out, float* nrm_out, cudaStream_t s) {
  SurfParams g;
  for (int a = 0; a < 3; ++a) g.lo[a] = h->lo[a];
  g.h = h->h;
  g.res = res;
  g.nb = div_up(res - 1, kBrick);
  const int nbricks = g.nb * g.nb * g.nb;
  int slot = stage_begin(h, kStMC, s);
  {
    // inside bits of the nodes (in the solver's idle correction buffer), then
    // the triangles per brick from them
    const int nw = div_up(res, 32);
    unsigned* bits = reinterpret_cast<unsigned*>(h->e32);
    mc_bits_kernel<<<dim3(nw, div_up((int64_t)res * res, 8 * kBitRows)), dim3(32, 8), 0, s>>>(h->chi32, res, nw,
                                                                                               h->dstate, bits);
    WGEO_LAUNCH_CHECK();
    const int64_t groups = (int64_t)div_up(res - 1, 32) * g.nb * g.nb;
    mc_count_kernel<<<grid_blocks(16 * groups, 256, h->num_sms * 16), 256, 0, s>>>(bits, g, nw, h->brick_count);
    WGEO_LAUNCH_CHECK();
  }
  int rc = exclusive_scan(h->brick_count, h->brick_off, nbricks, h->scan_tmp, s);
  if (rc) return rc;
  mc_total_kernel<<<1, 1, 0, s>>>(h->brick_off, nbricks, h->mesh_cap, h->leaf_off, h->dstate);
  WGEO_LAUNCH_CHECK();
  // the bricks with triangles, listed in the solver's idle residual buffer
  int* live_bricks = reinterpret_cast<int*>(h->r32);
  WGEO_CUDA_TRY(cudaMemsetAsync(&h->dstate->nbrick_live, 0, sizeof(unsigned), s));
  mc_live_kernel<<<grid_blocks(nbricks, 256, h->num_sms * 16), 256, 0, s>>>(h->brick_off, nbricks, h->leaf_off,
                                                                            live_bricks, &h->dstate->nbrick_live);
  WGEO_LAUNCH_CHECK();
  // vertices from the refined float-float indicator (MIXED precision) and
  // their low parts for the near-tie decisions and the adjoint (when kept)
  mc_emit_kernel<<<std::min(div_up(nbricks, kMcBricks), h->num_sms * 8), 64 * kMcBricks, 0, s>>>(
      h->chi32, chiff_of(h), g, h->dstate, h->brick_off, h->mesh_cap, live_bricks, &h->dstate->nbrick_live,
      h->tris, h->tris_lo, h->leaf_off, h->leaf_cnt);
  WGEO_LAUNCH_CHECK();
  const PyrInfo pi = pyramid_info(2 * g.nb);
  const int64_t nleaf = (int64_t)pi.dim[0] * pi.dim[0] * pi.dim[0];
  // the live leaves, listed in the correction buffer (its inside bits are consumed)
  int* live = reinterpret_cast<int*>(h->e32);
  WGEO_CUDA_TRY(cudaMemsetAsync(&h->dstate->nleaf_live, 0, sizeof(unsigned), s));
  puck_leaf_scan_kernel<<<grid_blocks(nleaf, 256, h->num_sms * 16), 256, 0, s>>>(h->leaf_off, g.nb, h->mesh_cap,
                                                                                 h->pyramid, live, h->dstate);
  WGEO_LAUNCH_CHECK();
  const int live_grid = grid_blocks(nleaf, 256, h->num_sms * 8);
  puck_leaf_kernel<<<live_grid, 256, 0, s>>>(h->tris, h->tris_lo, h->leaf_off, h->leaf_cnt, g.nb, h->mesh_cap, live,
                                             h->dstate, h->pyramid, h->tris_s, h->cell_pyr);
  WGEO_LAUNCH_CHECK();
  {
    // levels >= 1: sums per brick, sums up the tree, vertex maxima, pucks
    const int64_t nbr = (int64_t)g.nb * g.nb * g.nb;
    puck_sums_brick_kernel<<<grid_blocks(nbr, 128, 152 * 16), 128, 0, s>>>(h->tris, h->brick_off, g.nb,
                                                                           h->mesh_cap, h->pyr_sums, h->pyr_rth);
    WGEO_LAUNCH_CHECK();
    for (int l = 2; l < pi.nlev; ++l) {
      const int64_t np = (int64_t)pi.dim[l] * pi.dim[l] * pi.dim[l];
      puck_sums_up_kernel<<<grid_blocks(np, 128, 152 * 16), 128, 0, s>>>(
          h->pyr_sums, h->pyr_rth, pi.off[l - 1] - pi.off[1], pi.dim[l - 1], pi.off[l] - pi.off[1], pi.dim[l]);
      WGEO_LAUNCH_CHECK();
    }
    puck_rth_kernel<<<live_grid, 256, 0, s>>>(h->tris, h->leaf_off, g.nb, h->mesh_cap, pi, live, h->dstate,
                                              h->pyr_sums, h->pyr_rth);
    WGEO_LAUNCH_CHECK();
    const int64_t naux = pi.off[pi.nlev - 1] + 1 - pi.off[1];
    puck_finalize_kernel<<<grid_blocks(naux, 256, 152 * 16), 256, 0, s>>>(h->pyramid, h->pyr_sums, h->pyr_rth,
                                                                          naux, pi.off[1]);
    WGEO_LAUNCH_CHECK();
    puck_mask_kernel<<<grid_blocks(naux, 256, 152 * 16), 256, 0, s>>>(h->pyramid, pi);
    WGEO_LAUNCH_CHECK();
  }
  stage_end(h, kStMC, slot, s);
  slot = stage_begin(h, kStSDF, s);
  // the solver's residual / correction scratch is idle until the next solve:
  // it holds the near-tie candidates between the two kernels
  int* tie_a = reinterpret_cast<int*>(h->r32);
  int* tie_b = reinterpret_cast<int*>(h->e32);
  // ... and so does the float-float iterate buffer that is not the current one
  // (its index is on the device): two more candidates per node
  TieSlots tie_cd;
  tie_cd.p[0] = reinterpret_cast<int2*>(h->chiff[0]);
  tie_cd.p[1] = reinterpret_cast<int2*>(h->chiff[1]);
  int* ctri = h->opt.keep_for_backward ? h->ctri : nullptr;
  // closest triangles of the coarser passes, read by the finer ones as seeds
  int* seed_ids = ctri ? ctri : tie_a;
  // the near-tie list: nodes re-decided by the tie pass, in the adjoint's
  // dL/dchi buffer, which is idle until a backward clears it
  int* tie_list = ctri ? reinterpret_cast<int*>(h->dchi64) : nullptr;
  if (ctri) WGEO_CUDA_TRY(cudaMemsetAsync(&h->dstate->ntie, 0, sizeof(unsigned), s));
  // closest-feature keys of the near-tie candidates: the bits above the
  // triangle ids (ids < cap <= 2^id_bits - 1; at least 8 key bits)
  int id_bits = 0;
  if (ctri) {
    while (id_bits < 32 && ((int64_t)1 << id_bits) - 1 < h->mesh_cap) ++id_bits;
    if (id_bits > 24) id_bits = 0;
  }
  for (int stride = kSdfCoarse; stride >= 1; stride /= 2) {
    const int nl = (res + stride - 1) / stride;
    const int nblk = ((nl + 7) / 8) * ((nl + 7) / 8) * ((nl + 1) / 2);
    if (ctri) {
      if (h->opt.stage_timing == 2)
        sdf_kernel<true, true><<<nblk, kWarps * 32, 0, s>>>(h->chi32, g, h->dstate, h->tris_s, id_bits, h->leaf_off,
                                                            h->mesh_cap, h->pyramid, pi, h->phi, sdf_out, ctri,
                                                            tie_a, tie_b, tie_cd, tie_list, seed_ids, stride,
                                                            h->leaf_cnt, h->cell_pyr);
      else
        sdf_kernel<false, true><<<nblk, kWarps * 32, 0, s>>>(h->chi32, g, h->dstate, h->tris_s, id_bits, h->leaf_off,
                                                             h->mesh_cap, h->pyramid, pi, h->phi, sdf_out, ctri,
                                                             tie_a, tie_b, tie_cd, tie_list, seed_ids, stride,
                                                            h->leaf_cnt, h->cell_pyr);
    } else {
      if (h->opt.stage_timing == 2)
        sdf_kernel<true, false><<<nblk, kWarps * 32, 0, s>>>(h->chi32, g, h->dstate, h->tris_s, id_bits, h->leaf_off,
                                                             h->mesh_cap, h->pyramid, pi, h->phi, sdf_out, nullptr,
                                                             nullptr, nullptr, tie_cd, nullptr, seed_ids, stride,
                                                             h->leaf_cnt, h->cell_pyr);
      else
        sdf_kernel<false, false><<<nblk, kWarps * 32, 0, s>>>(h->chi32, g, h->dstate, h->tris_s, id_bits, h->leaf_off,
                                                              h->mesh_cap, h->pyramid, pi, h->phi, sdf_out, nullptr,
                                                              nullptr, nullptr, tie_cd, nullptr, seed_ids, stride,
                                                             h->leaf_cnt, h->cell_pyr);
    }
    WGEO_LAUNCH_CHECK();
  }
  stage_end(h, kStSDF, slot, s);
  if (ctri) {
    slot = stage_begin(h, kStSDFTie, s);
    sdf_tie_kernel<<<152 * 8, 256, 0, s>>>(h->chi32, g, h->dstate, h->tris_s, h->tris, h->tris_lo, tie_a, tie_b,
                                           tie_cd, tie_list, h->phi, sdf_out, ctri);
    WGEO_LAUNCH_CHECK();
    stage_end(h, kStSDFTie, slot, s);
  }
  if (nrm_out) {
    slot = stage_begin(h, kStNormals, s);
    normals_kernel<<<dim3(div_up(res, 32), div_up(res, 8), div_up(res, kNrmZ)), dim3(32, 8), 0, s>>>(
        h->phi, res, h->h, nrm_out);
    WGEO_LAUNCH_CHECK();
    stage_end(h, kStNormals, slot, s);
  }
  return WGEO_OK;
}

int launch_query_exact_chunk(wgeo_handle* h, const float* q, int nq, float* sdf_q, float* nrm_q, int* tri,
                             cudaStream_t s) {
  if (nq == 0) return WGEO_OK;
  SurfParams g;
  for (int a = 0; a < 3; ++a) g.lo[a] = h->lo[a];
  g.h = h->h;
  g.res = h->res;
  g.nb = div_up(h->res - 1, kBrick);
  const PyrInfo pi = pyramid_info(2 * g.nb);
  const int* ctri = h->opt.keep_for_backward ? h->ctri : nullptr;
  // queries sorted by (cell of 8 h, sub-cell key), so that a warp's 32
  // queries lie close together
  const float box[6] = {(float)g.lo[0], (float)g.lo[1], (float)g.lo[2], (float)(g.lo[0] + g.res * g.h),
                        (float)(g.lo[1] + g.res * g.h), (float)(g.lo[2] + g.res * g.h)};
  PointGrid pg;
  int rc = build_point_grid(h, q, nq, box, 8.0 * g.h, true, nullptr, &pg, s);
  if (rc) return rc;
  const int* total = h->dp_off + pg.ncell;
  const int nblk = grid_blocks((int64_t)nq, kWarps * 32, 152 * 8);
  if (ctri)
    sdf_query_kernel<true><<<nblk, kWarps * 32, 0, s>>>(h->phi, g, h->tris, h->tris_s, h->leaf_off, h->mesh_cap, h->pyramid,
                                                        pi, h->dp_sorted, total, ctri, sdf_q, nrm_q, tri);
  else
    sdf_query_kernel<false><<<nblk, kWarps * 32, 0, s>>>(h->phi, g, h->tris, h->tris_s, h->leaf_off, h->mesh_cap,
                                                         h->pyramid, pi, h->dp_sorted, total, nullptr, sdf_q, nrm_q,
                                                         tri);
  WGEO_LAUNCH_CHECK();
  query_sign_kernel<<<grid_blocks(nq, 128, 152 * 16), 128, 0, s>>>(q, nq, h->chi32, chiff_of(h), g, h->dstate,
                                                                    sdf_q, nrm_q);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

int launch_query_exact(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* nrm_q, cudaStream_t s) {
  // in chunks the point-grid workspace can sort
  for (int64_t c0 = 0; c0 < m; c0 += h->dp_points) {
    const int nq = (int)std::min<int64_t>(h->dp_points, m - c0);
    int rc = launch_query_exact_chunk(h, q + 3 * c0, nq, sdf_q + c0, nrm_q ? nrm_q + 3 * c0 : nullptr, nullptr, s);
    if (rc) return rc;
  }
  return WGEO_OK;
}

}  // namespace wgeo
