// Internal declarations shared by the library's translation units.
// Not part of the C ABI (include/wgeo.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/wgeo.h"

namespace wgeo {

// ---------------------------------------------------------------- constants
constexpr int kSplatTile = 8;        // output tile edge of the fused splat + divergence
constexpr int kBrick = 4;            // marching-cubes cubes per brick edge (SDF leaf)
constexpr int kMaxTriPerCube = 5;
constexpr int kTriRec = 4;           // float4 per triangle search record
constexpr int kMaxRes = 800;         // grid bound: packed coordinates, int32 edge ids and
                                     // 32-bit node indices stay in range
constexpr int kPartials = 2048;      // per-block partial slots of the deterministic reductions
constexpr int kMaxLevels = 12;
constexpr int kDpcaAxisCells = 1024;  // normal estimation: cells per axis at most
constexpr int kDpcaSub = 2;           // normal estimation: cell edge R / kDpcaSub (when the caps allow)
constexpr int kDpcaLanes = 4;         // normal estimation: lanes per point
constexpr int kDpcaPts = 32 / kDpcaLanes;   // points per warp chunk
constexpr int kDpcaBox = 16;          // sorted entries per bounding box
constexpr double kFixScale = 68719476736.0;      // 2^36: fixed-point scale of the splat sums
constexpr double kFixInv2 = 1.0 / 137438953472.0; // 1 / 2^37 (the face form sums 2 F)

// ---------------------------------------------------------------- device state
struct SolveState {
  int done;          // set once the relative residual is below tol (gates later kernels)
  int iter;          // refinement steps / V-cycles performed
  int xidx;          // which of the two FP64 buffers holds the current iterate
  int cold;          // 1: start from x = 0 (the first refinement pass writes zeros)
  int max_steps;     // the last step allowed (refinement steps, or V-cycles in plain FP32)
  int min_steps;     // the first step that may stop (2 with the spectral correction, else 0)
  int body_launches; // kernels of one iteration of the recorded loop body (launch accounting)
  double bnorm;      // || b - mean(b) ||
  double bmean;
  double rmean;      // mean of the last residual (projected out of the correction RHS)
  float bmean32;     // the two means rounded to float once, for the FP32 kernels
  float rmean32;
  double rel;        // last || r || / || b ||
};

struct DevState {
  unsigned int status;
  int pad0;
  long long npts;     // finite points used by the forward
  long long ntris;    // triangles found (uncapped)
  double c;           // iso-value
  float c_up;         // the smallest float >= c: for float chi, chi < c <=> chi < c_up
  double dc;          // backward: dL/dc
  SolveState fwd;
  SolveState bwd;
  unsigned long long sdf_cnt[4];   // octree nodes entered, leaves entered, lane point-triangle tests,
                                   // nodes re-decided in float-float
  unsigned nsliver;                // backward: nodes whose closest triangle is a sliver (FP64 pass)
  unsigned ntie;                   // forward: nodes on the near-tie list (distance search)
  unsigned splat_tiles;            // forward: splat tiles with a point in reach (the active list)
  unsigned splat_next;             // forward: next active tile to be taken by a splat CTA
  unsigned nleaf_live;             // forward: octree leaves holding triangles (the live list)
  unsigned nbrick_live;            // forward: marching-cubes bricks holding triangles (the live list)
  unsigned nmax_bits;              // forward: largest |normal component| of the points (float bits)
};

struct Tri {          // one marching-cubes triangle: vertex xyz + global edge id in .w
  float4 a, b, c;
};

// The two float-float indicator buffers of the forward solve (refinement
// ping-pong; DevState::fwd.xidx selects the current one), or null pointers
// when the handle solves in plain FP32.
struct ChiFF {
  const float2* p[2];
};

struct Level {
  int n;
  float* x;
  float* b;
  float* t;   // Jacobi ping-pong buffer (unlumped Galerkin operator only)
};

// Unlumped trilinear Galerkin operator, scaled by 12 so that its weights are
// integers: (L' x)_p = sum over the 12 edge neighbours of 2 (x_q - x_p) plus
// the 8 corner neighbours of (x_q - x_p) (the 6 face neighbours have weight
// 0), the walls mirrored (an index outside the grid folds onto the cell
// inside).  12 times the unit-free form -(S M M + M S M + M M S).
constexpr int kQ1Scale = 12;

// ---------------------------------------------------------------- stage timers
// Stage ids of the per-stage CUDA-event timers (option stage_timing).
enum Stage {
  kStSplat = 0,    // bin + tile sort + fused splat/divergence
  kStSolve = 1,    // forward Poisson solve
  kStIso = 2,
  kStMC = 3,       // count + scan + emit + box pyramid
  kStSDF = 4,      // exact distance search + sign
  kStNormals = 5,
  kStQuery = 6,
  kStBwdSeed = 7,  // grid seeds + query adjoint
  kStBwdSurf = 8,  // distance / marching-cubes / iso-value adjoints
  kStBwdSolve = 9,
  kStBwdSplat = 10,
  kStSDFTie = 11,  // near-tie decisions of the distance search
  kStPointPca = 12,  // D-PCA normal estimation
  kStOrient = 13,    // parity orientation
  kStQueryExact = 14,  // exact off-grid signed distance
  kStages = 15
};
constexpr int kRing = 256;

struct StageTimer {
  cudaEvent_t beg[kRing];
  cudaEvent_t end[kRing];
  bool used[kRing];
  int head = 0;
  double acc_ms = 0.0;
  long long count = 0;
};

// ---------------------------------------------------------------- handle
struct SolverGraph {
  int res = 0;
  int mode = -1;      // 0 forward, 1 backward
  long long launches = 0;       // kernels of the graph's head (run once per replay)
  long long body_launches = 0;  // kernels of one iteration of its device-side loop
  cudaGraphExec_t exec = nullptr;
};

// ---- float-float arithmetic (value = x + y, |y| <= ulp(x)/2).  Knuth's
// two-sum and Dekker's fast two-sum give the exact rounding error of one
// addition; the __f*_rn intrinsics keep the compiler from contracting or
// reordering them.
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, err);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {   // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  const float2 t = two_sum(a.y, b.y);
  const float2 r = fast_two_sum(s.x, __fadd_rn(s.y, t.x));
  return fast_two_sum(r.x, __fadd_rn(r.y, t.y));
}
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 ff_add_f(float2 a, float b) {
  const float2 s = two_sum(a.x, b);
  return fast_two_sum(s.x, __fadd_rn(s.y, a.y));
}

// Node coordinate u = (x - lo) / h - 1/2 of a float position along one axis,
// in float-float (x - lo by two-sum, the product with 1/h from its exact FMA
// residual): about 2^-44 relative, so floor(u) and the fraction are those of
// the exact quotient up to the fraction's final float rounding, with no FP64
// arithmetic (lo and 1/h come as float-float pairs).
__device__ __forceinline__ float2 node_coord_ff(float x, float lo_hi, float lo_lo, float ih_hi, float ih_lo) {
  float2 d = two_sum(x, -lo_hi);
  d = fast_two_sum(d.x, __fsub_rn(d.y, lo_lo));
  const float ph = __fmul_rn(d.x, ih_hi);
  const float pl = __fadd_rn(__fmaf_rn(d.x, ih_hi, -ph), __fadd_rn(__fmul_rn(d.x, ih_lo), __fmul_rn(d.y, ih_hi)));
  const float2 u = fast_two_sum(ph, pl);
  const float2 um = two_sum(u.x, -0.5f);
  return fast_two_sum(um.x, __fadd_rn(um.y, u.y));
}

// Cell and fraction of a float-float node coordinate clamped to [0, top]
// (top = n - 1): f = min(floor u, n - 2), t = u - f.  Returns whether u was
// clamped.
__device__ __forceinline__ bool node_cell_ff(float2 u, int n, int& f, float& t) {
  const float top = (float)(n - 1);
  const bool below = u.x < 0.f || (u.x == 0.f && u.y < 0.f);
  const bool above = u.x > top || (u.x == top && u.y > 0.f);
  if (below) u = make_float2(0.f, 0.f);
  if (above) u = make_float2(top, 0.f);
  float fl = floorf(u.x);
  if (u.x == fl && u.y < 0.f) fl -= 1.f;
  f = min((int)fl, n - 2);
  t = __fadd_rn(__fsub_rn(u.x, (float)f), u.y);
  return below || above;
}

// A double as hi + lo floats without the FP64 pipe (integer and FP32 work
// only; the FP64 pipe of this GPU is a small fraction of its FP32 rate):
// hi keeps the top 24 significand bits (truncated), lo the other 29 rounded
// to float, so hi + lo equals v to 2^-47 relative, as a rounded pair does.  Zero and
// FP64 subnormals give (signed zero, 0); magnitudes outside [2^-74, 2^127)
// take the FP64 conversions.
__device__ __forceinline__ float2 split_f64(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hw = (unsigned)(u >> 32);
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e == 0) return make_float2(__uint_as_float(sign), 0.f);
  if (e < 949 || e > 1150) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  }
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((u >> 29) & 0x7fffffull));
  const float lo = __uint2float_rn((unsigned)(u & 0x1fffffffull)) * __uint_as_float((unsigned)(e - 948) << 23);
  return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ float3 f3(const float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Float-float scalar (about 44 significant bits on the FP32 pipe) for the
// near-tie decisions of the distance search: sums by two-sum, products with
// the FMA residual (fma(a, b, -rn(a b)) is the exact error of the rounded
// product).  Comparisons are exact for normalised values (|lo| <= ulp(hi) /
// 2), which every operator returns.
struct Ff {
  float hi, lo;
  __device__ __forceinline__ Ff() {}
  __device__ __forceinline__ Ff(float x) : hi(x), lo(0.f) {}
  __device__ __forceinline__ Ff(float h, float l) : hi(h), lo(l) {}
};
__device__ __forceinline__ Ff operator+(Ff a, Ff b) {
  const float2 r = ff_add(make_float2(a.hi, a.lo), make_float2(b.hi, b.lo));
  return Ff(r.x, r.y);
}
__device__ __forceinline__ Ff operator-(Ff a) { return Ff(-a.hi, -a.lo); }
__device__ __forceinline__ Ff operator-(Ff a, Ff b) { return a + (-b); }
__device__ __forceinline__ Ff operator*(Ff a, Ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float2 r = fast_two_sum(p, e);
  return Ff(r.x, r.y);
}
__device__ __forceinline__ bool operator<(Ff a, Ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(Ff a, Ff b) { return b < a; }
__device__ __forceinline__ bool operator<=(Ff a, Ff b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(Ff a, Ff b) { return !(a < b); }

// Closest-point weights (v, w) of y = a + v ab + w ac on a triangle given by
// its search record (r0 = (a, |ab|^2), r1 = (ab, vertex keys), r2 = (ac, |ac|^2),
// r3 = (1/|ab|^2, 1/|ac|^2, 1/|bc|^2, 1/|ab x ac|^2)), from ap = p - a,
// d1 = ab.ap and d2 = ac.ap: Ericson's Voronoi-region case analysis with the
// six dot products reduced to two through the Gram entries and the
// divisions replaced by the reciprocals.
__device__ __forceinline__ void rec_weights(const float3 ap, float d1, float d2, const float4 r0, const float4 r1,
                                            const float4 r2, const float4 r3, float& v, float& w) {
  const float e00 = r0.w, e01 = r1.x * r2.x + r1.y * r2.y + r1.z * r2.z, e11 = r2.w;   // r1.w: vertex keys
  const float d3 = d1 - e00, d4 = d2 - e01;                  // ab . bp, ac . bp
  const float d5 = d1 - e01, d6 = d2 - e11;                  // ab . cp, ac . cp
  if (d1 <= 0.f && d2 <= 0.f) {
    v = 0.f; w = 0.f;                                          // vertex a
  } else if (d3 >= 0.f && d4 <= d3) {
    v = 1.f; w = 0.f;                                          // vertex b
  } else {
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
      v = d1 * r3.x; w = 0.f;                                  // edge ab
    } else if (d6 >= 0.f && d5 <= d6) {
      v = 0.f; w = 1.f;                                        // vertex c
    } else {
      const float vb = d5 * d2 - d1 * d6;
      if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        v = 0.f; w = d2 * r3.y;                                // edge ac
      } else {
        const float va = d3 * d6 - d5 * d4;
        if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
          w = (d4 - d3) * r3.z; v = 1.f - w;                   // edge bc
        } else if (r3.w > 0.f) {
          v = vb * r3.w; w = vc * r3.w;                        // face
        } else {
          // collapsed triangle: the nearest of its three vertices
          const float qa = ap.x * ap.x + ap.y * ap.y + ap.z * ap.z;
          const float qb = qa - 2.f * d1 + e00, qc = qa - 2.f * d2 + e11;
          v = (qb < qa && qb <= qc) ? 1.f : 0.f;
          w = (qc < qa && qc < qb) ? 1.f : 0.f;
        }
      }
    }
  }
}

// Closest point y = wa a + wb b + wc c of triangle (a, b, c) to p in FP64:
// the face point when the projection falls inside (2 x 2 normal equations),
// else the nearest of the three edge points (segments clamped); returns
// |p - y|^2 and the unit direction (p - y) / |p - y| (zero when p is on the
// triangle).  For the rare ill-conditioned (sliver) triangles, where float32
// barycentric weights lose their digits while the distance does not.
__device__ __forceinline__ double closest_point_fp64(const double p[3], const double a[3], const double b[3],
                                                     const double c[3], double bw[3], double dir[3]) {
  double ab[3], ac[3], ap[3];
  for (int k = 0; k < 3; ++k) {
    ab[k] = b[k] - a[k];
    ac[k] = c[k] - a[k];
    ap[k] = p[k] - a[k];
  }
  auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
  double best = -1.0;
  double bv = 0.0, bwv = 0.0;   // weights of b and c
  const double d00 = dot(ab, ab), d01 = dot(ab, ac), d11 = dot(ac, ac);
  const double r0 = dot(ab, ap), r1 = dot(ac, ap);
  const double det = d00 * d11 - d01 * d01;
  if (det > 0.0) {
    const double v = (d11 * r0 - d01 * r1) / det, w = (d00 * r1 - d01 * r0) / det;
    if (v >= 0.0 && w >= 0.0 && v + w <= 1.0) {
      double r[3];
      for (int k = 0; k < 3; ++k) r[k] = ap[k] - v * ab[k] - w * ac[k];
      best = dot(r, r);
      bv = v;
      bwv = w;
    }
  }
  if (best < 0.0) {
    // edges ab (v = t), ac (w = t), bc (v = 1 - t, w = t)
    const double* P0[3] = {a, a, b};
    const double* P1[3] = {b, c, c};
    for (int e = 0; e < 3; ++e) {
      double d[3], q[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = P1[e][k] - P0[e][k];
        q[k] = p[k] - P0[e][k];
      }
      const double L2 = dot(d, d);
      double t = L2 > 0.0 ? dot(q, d) / L2 : 0.0;
      t = fmin(fmax(t, 0.0), 1.0);
      double r[3];
      for (int k = 0; k < 3; ++k) r[k] = q[k] - t * d[k];
      const double dd = dot(r, r);
      if (best < 0.0 || dd < best) {
        best = dd;
        bv = e == 0 ? t : (e == 2 ? 1.0 - t : 0.0);
        bwv = e == 1 ? t : (e == 2 ? t : 0.0);
      }
    }
  }
  bw[0] = fmax(1.0 - bv - bwv, 0.0);
  bw[1] = bv;
  bw[2] = bwv;
  double y[3], r[3];
  for (int k = 0; k < 3; ++k) {
    y[k] = bw[0] * a[k] + bw[1] * b[k] + bw[2] * c[k];
    r[k] = p[k] - y[k];
  }
  const double len = sqrt(dot(r, r));
  for (int k = 0; k < 3; ++k) dir[k] = len > 0.0 ? r[k] / len : 0.0;
  return best;
}

// |ab|^2 |ac|^2 / |ab x ac|^2 (1 / sin^2 of the angle at a) from a search
// record: above this the float32 weights are replaced by closest_point_fp64.
constexpr float kSliverKappa = 1e3f;

template <typename T>
struct Vec3 {
  T x, y, z;
};


}  // namespace wgeo

struct wgeo_handle {
  int max_res = 0;
  int64_t max_points = 0;
  wgeo_options opt{};
  int device = 0;
  int num_sms = 1;   // the device's multiprocessor count (grids of persistent kernels)

  // arena
  char* arena = nullptr;
  size_t arena_bytes = 0;

  // grid fields (sized for max_res^3)
  float* b32 = nullptr;
  float* chi32 = nullptr;
  float2* chiff[2] = {nullptr, nullptr};   // float-float iterate, ping-pong (index on the device)
  float* r32 = nullptr;
  float* e32 = nullptr;
  float* phi = nullptr;
  int* ctri = nullptr;
  float* dphi = nullptr;         // backward: dL/dphi per node (float: its atomics stay in L2)
  double* dchi64 = nullptr;
  float2* lamff[2] = {nullptr, nullptr};   // adjoint solution, ping-pong like chiff
  float* lam32 = nullptr;
  float* level_pool = nullptr;
  // spectral solve tables for n = 32 R (the lane layout: entry a * 32 + j for lane j, register a)
  float2* dct_t1 = nullptr;      //   e^{-2 pi i j a / n} (a < R)
  float2* dct_w32 = nullptr;     //   per lane-butterfly stage s (h = 2^s): e^{-i pi (j mod h) / h}
  float2* dct_wml = nullptr;     //   e^{-i pi k / (2 n)} at k = a + R brev5(j)
  float2* dct_tr = nullptr;      //   e^{-2 pi i q / R} (q < R)
  float2* dct_tw = nullptr;      //   e^{-2 pi i q / n} (q < n)
  float2* dct_wq = nullptr;      //   e^{-i pi q / (2 n)} (q <= n)
  float* dct_sk = nullptr;       //   4 sin^2(pi k / (2 n)) (k < n, natural order)
  float* dct_skl = nullptr;      //   the same at k = a + R brev5(j)
  int dct_n = 0;                 // n the tables hold (0: none yet)
  bool dct_attr = false;         // shared-memory opt-in of the pass kernels done (per device)

  // points
  int* pcell = nullptr;          // packed central cell per point (original order); -1 = skipped
  float4* pfrac = nullptr;       // (u - cell) per axis, original order
  float4* pnrm = nullptr;        // copy of the normals, original order (backward)
  float4* srec = nullptr;        // sorted records: 2 float4 per point
  int* tile_count = nullptr;
  int* tile_off = nullptr;       // ntiles + 1
  int* tile_cursor = nullptr;

  // mesh
  int64_t mesh_cap = 0;
  int* brick_count = nullptr;
  int* brick_off = nullptr;      // nbricks + 1
  int* leaf_off = nullptr;       // 8 * nbricks + 1: triangle offset of each 2^3 sub-brick
  unsigned* leaf_cnt = nullptr;  // 8 * nbricks: the triangle counts of a sub-brick's 8 cubes, 4 bits each
  wgeo::Tri* tris = nullptr;
  wgeo::Tri* tris_lo = nullptr;  // keep_for_backward: per vertex the low part of its ~48-bit position
                                 // (FP64 vertex - float32 vertex); null otherwise
  float4* tris_s = nullptr;      // per triangle: search record (a, |ab|^2), (ab, ab.ac), (ac, |ac|^2),
                                 // (1/|ab|^2, 1/|ac|^2, 1/|bc|^2, 1/|ab x ac|^2)
  float4* pyramid = nullptr;     // 2 float4 per node (puck: centre + radius, axis + half-thickness)
  float4* cell_pyr = nullptr;    // per cube with triangles: its puck, at the slot of its first triangle
  float4* pyr_sums = nullptr;    // levels >= 1: vertex sum + count, area-normal sum (puck construction)
  unsigned* pyr_rth = nullptr;   // levels >= 1: radius, half-thickness as float bits (atomic maxima)
  double* dP = nullptr;          // backward: dL/d(vertex) per triangle corner, 9 doubles

  // normal estimation (its own buffers: a call between a forward and its
  // backward leaves the forward's state intact)
  int64_t dp_cell_cap = 0;       // cells the workspace holds
  int64_t dp_points = 0;         // points it holds (exact queries are sorted in chunks of this size)
  int* dp_cell = nullptr;        // cell per point (original order); -1 = non-finite
  int* dp_count = nullptr;       // dp_cell_cap + 1
  int* dp_off = nullptr;         // dp_cell_cap + 2 (exclusive scan, total last)
  int* dp_cursor = nullptr;      // dp_cell_cap + 1 (after the call's cells: the chunk counter)
  int* dp_key = nullptr;         // sub-cell key per grouped entry
  float4* dp_gbox = nullptr;     // 2 float4 per kDpcaBox sorted entries: bounding box
  unsigned* or_scal = nullptr;   // orientation: cloud box (ordered bits), max nearest distance^2
  int* dp_scan = nullptr;
  float4* dp_tmp = nullptr;      // points grouped by cell, unordered within a cell
  float4* dp_sorted = nullptr;   // the same, point-index order within each cell

  // reductions / scans
  double* partials = nullptr;    // kPartials * 4 doubles
  int* scan_tmp = nullptr;
  size_t scan_tmp_elems = 0;

  wgeo::DevState* dstate = nullptr;

  // host-side state of the last forward
  int res = 0;
  double h = 0.0;
  double lo[3] = {0, 0, 0};
  int64_t npts = 0;
  bool have_forward = false;
  bool have_backward_state = false;
  bool chi_valid_for_warm = false;
  int warm_res = 0;
  cudaStream_t last_stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  wgeo::SolverGraph graphs[4];   // [2 mode + (the cold head skipped)]

  // multigrid hierarchy for the current res
  int nlevels = 0;
  wgeo::Level levels[wgeo::kMaxLevels];

  // per-stage event timers (allocated on first use when opt.stage_timing is set)
  wgeo::StageTimer* timers = nullptr;
  int bwd_slot = -1;             // timer slot of the backward's surface stage
};

namespace wgeo {
// The forward's float-float indicator buffers when the handle refines its
// solve (MIXED, or FP64 whose iterate is converted to a float-float pair after
// the solve): vertex placement, near-tie decisions, sign tests and the
// adjoint's vertex weights read the current one.  Null pointers in FP32 mode.
inline ChiFF chiff_of(const wgeo_handle* h) {
  ChiFF c;
  const bool mixed = h->opt.precision != WGEO_PREC_FP32;
  c.p[0] = mixed ? h->chiff[0] : nullptr;
  c.p[1] = mixed ? h->chiff[1] : nullptr;
  return c;
}

// Records the start / end of a stage on stream s (no-ops unless stage timing is on).
int stage_begin(wgeo_handle* h, int stage, cudaStream_t s);
void stage_end(wgeo_handle* h, int stage, int slot, cudaStream_t s);
}  // namespace wgeo

namespace wgeo {

// ---------------------------------------------------------------- helpers
#define WGEO_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return WGEO_ERR_CUDA;              \
  } while (0)

// Kernel launches enqueued by this library (process-wide, and per host thread
// so that a stream capture can tell its own launches apart).  Every launch is
// followed by exactly one WGEO_LAUNCH_CHECK, which counts it.
extern std::atomic<long long> g_kernel_launches;
extern thread_local long long t_kernel_launches;

#define WGEO_LAUNCH_CHECK()                                   \
  do {                                                        \
    ::wgeo::g_kernel_launches.fetch_add(1, std::memory_order_relaxed); \
    ++::wgeo::t_kernel_launches;                              \
    cudaError_t _e = cudaGetLastError();                      \
    if (_e != cudaSuccess) return WGEO_ERR_CUDA;              \
  } while (0)

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int grid_blocks(int64_t n, int threads, int cap = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// coarsest-level rule: halve while even and larger than 8
int coarsest_size(int res);
long long loop_launches();   // kernels run by recorded solver loops on the current device (syncs)
int build_levels(wgeo_handle* h, int res);

// ---------------------------------------------------------------- launchers
// splat.cu
int launch_bin_sort_splat(wgeo_handle* h, const float* points, const float* normals, int64_t n,
                          int res, cudaStream_t s);
int launch_unpack_bins(wgeo_handle* h, int* out, cudaStream_t s);
// solver.cu
int launch_solve(wgeo_handle* h, int res, int mode, bool cold, cudaStream_t s);
// surface.cu
int launch_isovalue(wgeo_handle* h, const float* points, int64_t n, int res, cudaStream_t s);
int launch_mc_sdf_normals(wgeo_handle* h, int res, float* sdf_out, float* nrm_out, cudaStream_t s);
int upload_mc_table();
size_t pyramid_nodes(int nb);
size_t pyramid_aux_nodes(int nb);   // nodes of the levels above the leaves
void host_mc_table(int* counts, int* tris);
// query.cu
int launch_query(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* nrm_q, cudaStream_t s);
// surface.cu: exact signed distance and its gradient at arbitrary points
int launch_query_exact(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* nrm_q, cudaStream_t s);
// one chunk of at most dp_points queries; tri (may be NULL) receives the closest triangles
int launch_query_exact_chunk(wgeo_handle* h, const float* q, int nq, float* sdf_q, float* nrm_q, int* tri,
                             cudaStream_t s);
// query.cu: the backward with seeds of exact queries
int launch_backward_exact(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                          const float* d_sdf_q, int64_t m, float* d_points, float* d_normals, float* d_q,
                          cudaStream_t s);
int launch_export_adjoint(wgeo_handle* h, int which, float* out, cudaStream_t s);
int launch_backward(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                    const float* d_sdf_q, const float* d_nrm_q, int64_t m, float* d_points,
                    float* d_normals, float* d_q, cudaStream_t s);
// dpca.cu: point grids (cubic cells over a box; points outside it fall in the
// edge cells), built into the handle's normal-estimation workspace.  ordered:
// entries by (cell, sub-cell key, index) in dp_sorted; else by cell only,
// in arrival order, also in dp_sorted.
struct PointGrid {
  float lo[3];
  float inv_cs;   // 1 / cell edge
  int dim[3];
  int ncell;
  double cs;      // cell edge
};
int64_t point_grid_cap(int64_t max_points);
int point_grid_dims(const float* bbox, double cs_min, int64_t n, int64_t cap_ws, PointGrid* g);
int build_point_grid(wgeo_handle* h, const float* points, int n, const float* bbox, double cs_min, bool ordered,
                     float* zero_normals, PointGrid* g, cudaStream_t s);
int launch_dpca(wgeo_handle* h, const float* points, int64_t n, const float* bbox, float radius, float eps,
                float* normals, int* counts, cudaStream_t s);
// orient.cu
int launch_orient(wgeo_handle* h, const float* points, int64_t n, const float* bbox, float gamma, int n_tol,
                  float* normals, int* stats, float* rd_out, cudaStream_t s);
// scan.cu
int exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s);
size_t scan_tmp_size(int n);
// shgen.cu
int launch_sh_surface(const float* theta, int K, const float* dirs, int64_t n, float base,
                      const float* centre, float* points, float* normals, cudaStream_t s);
int launch_sh_backward(wgeo_handle* h, const float* theta, int K, const float* dirs, int64_t n,
                       float base, const float* dpts, const float* dnrm, float* dtheta, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sumi(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed shuffle tree, fixed warp order); result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (l < NT / 32) ? sh[l] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// Cell of a point in a PointGrid, clamped into the grid (float clamp before
// the conversion, so far points land in the edge cells).
__device__ __forceinline__ void grid_cell3(const PointGrid& g, float x, float y, float z, int c[3]) {
  const float p[3] = {x, y, z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float u = fminf(fmaxf(floorf((p[a] - g.lo[a]) * g.inv_cs), 0.f), (float)(g.dim[a] - 1));
    c[a] = (int)u;
  }
}
__device__ __forceinline__ int grid_cell(const PointGrid& g, float x, float y, float z) {
  int c[3];
  grid_cell3(g, x, y, z, c);
  return (c[2] * g.dim[1] + c[1]) * g.dim[0] + c[0];
}

__device__ __forceinline__ int pack_cell(int x, int y, int z) { return x | (y << 10) | (z << 20); }
__device__ __forceinline__ int cell_x(int p) { return p & 1023; }
__device__ __forceinline__ int cell_y(int p) { return (p >> 10) & 1023; }
__device__ __forceinline__ int cell_z(int p) { return (p >> 20) & 1023; }

}  // namespace wgeo
