// Poisson solve A a = b (Sec. 2.3, Eqs. 15, 20-21; adjoint solve Eq. 38).
//
// Operator: unit-free cell-centred 7-point Neumann Laplacian
//   (L x)_p = sum over in-grid neighbours q of (x_q - x_p),
// the transverse-lumped trilinear Galerkin stiffness (up to sign and a factor
// h).  The system is singular (constants) and consistent after projecting the
// mean out of the right-hand side; chi is defined up to an additive constant.
//
// Mixed precision (default): iterative refinement in double-float around FP32
//   multigrid.  The iterate is a float-float pair (hi + lo, ~48-bit
//   significand, error-free two-sum arithmetic on the FP32 pipe; this GPU's
//   FP64 pipe made a native FP64 residual pass ~12x slower than its memory
//   traffic).  One fused pass per refinement step adds the last FP32
//   correction (ping-pong buffers selected by a device-side index, so early
//   exit needs no host decision), writes the FP32 copy and the residual
//   r = b - L x, and sums r and r^2 (FP64 across threads and blocks); a
//   one-block kernel reduces the sums in a fixed order and tests
//   ||r - mean r|| <= tol ||b - mean b||.  The correction solves
//   L e = r - mean(r) with FP32 V-cycles.
// Plain FP32 (comparator): no refinement.  On power-of-two grids (with the
//   spectral option) one direct FP32 spectral solve of L x = b - mean(b);
//   elsewhere FP32 V-cycles directly on x32.  The residual and its norms are
//   FP32.
//
// Multigrid: cell-centred, halving while even and larger than 8; red-black
// Gauss-Seidel, 2 pre- and 2 post-sweeps; residual restricted with weight 1/2
// on the 8 children (average x H^2/h^2 for the unit-free operator); trilinear
// prolongation (3/4, 1/4 per axis, mirrored at the walls).  Levels above 16^3
// run one plain kernel per half-sweep, restriction and prolongation, each
// near its memory floor; grids of at most 16^3 run a whole V-cycle hierarchy
// in one CTA's shared memory.
//
// A solve is recorded once as a CUDA graph: the first residual and
// convergence test, then a conditional WHILE node whose body (one correction,
// residual and test) repeats until the test clears the condition, at the
// latest after the last allowed step; nothing is launched after convergence.
// Without graphs (or under the caller's own capture) the same kernels run as
// a fixed sequence of the allowed steps, each returning at once once the
// solve's `done` flag is set.
#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

constexpr int kThreads = 256;
constexpr int kSX = 32, kSY = 8;    // 3D-grid blocks: 32 x pairs by 8 rows of one plane
constexpr int kNu = 2;              // red-black sweeps before and after the coarse correction
constexpr int kSmallN = 16;         // levels up to 16^3 are solved in one CTA

__device__ __forceinline__ int64_t lin(int i, int j, int k, int n) {
  return ((int64_t)k * n + j) * n + i;
}

struct PairFF {
  float2* buf[2];
};
struct PairD {
  double* buf[2];
};

__device__ __forceinline__ float rhs_hi(const float* b, int64_t t, float& lo) {
  lo = 0.f;
  return b[t];
}
__device__ __forceinline__ float rhs_hi(const double* b, int64_t t, float& lo) {
  const float2 p = split_f64(b[t]);
  lo = p.y;
  return p.x;
}

// ---------------------------------------------------------------- refinement pass
// The refinement iterate is kept in float-float (hi + lo, ~48-bit significand):
// on this GPU the FP64 pipe made an FP64 stencil pass about 12x slower than its
// memory traffic, while the error-free sums below run on the FP32 pipe.
//   x_new = x + e (e may be null: no correction this step; cold: x := 0),
//   x32 = hi(x_new), r32 = b - L x_new (each neighbour difference split
//   exactly), per-thread sums of r and r^2 in FP32, per-block sums in FP64.
// One x pair (i0 = 2 I, i0 + 1) of row j per thread, marching kResZ planes in
// z: the pair's x_new below, at and above the current plane stay in
// registers, so only the plane above is loaded per step (with the y
// neighbours' pairs and the two x neighbours).  The neighbour differences
// are summed in the same order as a one-plane-per-thread pass (x partner,
// x - 1, x + 2, y - 1, y + 1, z - 1, z + 1), so x32 and r32 do not depend on
// the marching.
constexpr int kResZ = 8;
template <typename TB>
__global__ void __launch_bounds__(kSX * kSY, 4) update_residual_kernel(PairFF xp, const float* __restrict__ e,
                                                                    const TB* __restrict__ b, int n,
                                                                    float* __restrict__ r32, float* __restrict__ x32,
                                                                    double* __restrict__ partials, SolveState* ss) {
  if (ss->done) return;
  __shared__ double red[2 * (kSX * kSY / 32)];
  const int cur = ss->xidx;
  const bool cold = ss->cold != 0;
  const float2* __restrict__ xin = xp.buf[cur];
  float2* __restrict__ xout = xp.buf[e ? cur ^ 1 : cur];
  // vector accesses need an even n (pairs then start on even cells); an odd
  // n (only grids up to 15^3) takes scalar accesses and a last pair of one cell
  const int I = blockIdx.x * kSX + threadIdx.x, j = blockIdx.y * kSY + threadIdx.y;
  const int k0 = blockIdx.z * kResZ, k1 = min(k0 + kResZ, n);
  const int i0 = 2 * I;
  const bool vec = (n & 1) == 0;
  float s1 = 0.f, s2 = 0.f;
  if (i0 < n && j < n) {
    const bool has1 = i0 + 1 < n;
    const int64_t nn = (int64_t)n * n;
    // a cold start reads x as 0: with no correction x_new = 0 and r = b; with
    // one (the first iteration of a solve without a head) x_new = e
    const bool stencil = !cold || e;
    auto pair = [&](int64_t q, float2& a, float2& c) {   // x_new at cells q, q + 1
      if (vec) {
        const float4 v = cold ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(xin + q);
        a = make_float2(v.x, v.y);
        c = make_float2(v.z, v.w);
        if (e) {
          const float2 ev = *reinterpret_cast<const float2*>(e + q);
          a = ff_add_f(a, ev.x);
          c = ff_add_f(c, ev.y);
        }
      } else {
        a = cold ? make_float2(0.f, 0.f) : xin[q];
        if (e) a = ff_add_f(a, e[q]);
        c = make_float2(0.f, 0.f);
        if (has1) {
          c = cold ? make_float2(0.f, 0.f) : xin[q + 1];
          if (e) c = ff_add_f(c, e[q + 1]);
        }
      }
    };
    auto single = [&](int64_t q) {
      const float2 v = cold ? make_float2(0.f, 0.f) : xin[q];
      return e ? ff_add_f(v, e[q]) : v;
    };
    const float2 zero2 = make_float2(0.f, 0.f);
    // x_new of the pair on planes k - 1 (zm), k (zc) and k + 1 (zp)
    float2 zm[2] = {zero2, zero2}, zc[2] = {zero2, zero2}, zp[2] = {zero2, zero2};
    int64_t t0 = (int64_t)k0 * nn + (int64_t)j * n + i0;
    if (stencil) {
      if (k0 > 0) pair(t0 - nn, zm[0], zm[1]);
      pair(t0, zc[0], zc[1]);
    }
    for (int k = k0; k < k1; ++k, t0 += nn) {
      float2 acc[2] = {zero2, zero2};
      if (stencil) {
        if (k < n - 1) pair(t0 + nn, zp[0], zp[1]);
        // L x = sum of (x_q - x_p): each hi difference split exactly by two-sum,
        // the hi parts summed by a two-sum chain (rounding errors carried in
        // `err`), the lo differences (each below ulp(hi)) summed in float
        float sh[2] = {0.f, 0.f}, err[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
        auto add = [&](int c, float2 v) {
          const float2 d = two_sum(v.x, -zc[c].x);
          const float2 q = two_sum(sh[c], d.x);
          sh[c] = q.x;
          err[c] = __fadd_rn(err[c], __fadd_rn(q.y, d.y));
          lo[c] = __fadd_rn(lo[c], __fsub_rn(v.y, zc[c].y));
        };
        if (has1) {
          add(0, zc[1]);                     // the pair's own cells are x neighbours
          add(1, zc[0]);
        }
        if (i0 > 0) add(0, single(t0 - 1));
        if (i0 + 2 < n) add(1, single(t0 + 2));
        float2 a, c;
        if (j > 0) { pair(t0 - n, a, c); add(0, a); add(1, c); }
        if (j < n - 1) { pair(t0 + n, a, c); add(0, a); add(1, c); }
        if (k > 0) { add(0, zm[0]); add(1, zm[1]); }
        if (k < n - 1) { add(0, zp[0]); add(1, zp[1]); }
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[q] = two_sum(sh[q], __fadd_rn(err[q], lo[q]));
      }
      float rf[2] = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 1 && !has1) break;
        float blo;
        const float bhi = rhs_hi(b, t0 + q, blo);
        const float2 r = ff_sub(make_float2(bhi, blo), acc[q]);
        rf[q] = r.x + r.y;
        s1 += rf[q];
        s2 += rf[q] * rf[q];
      }
      if (vec) {
        if (e || cold) *reinterpret_cast<float4*>(xout + t0) = make_float4(zc[0].x, zc[0].y, zc[1].x, zc[1].y);
        *reinterpret_cast<float2*>(x32 + t0) = make_float2(zc[0].x, zc[1].x);
        *reinterpret_cast<float2*>(r32 + t0) = make_float2(rf[0], rf[1]);
      } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q == 1 && !has1) break;
          if (e || cold) xout[t0 + q] = zc[q];
          x32[t0 + q] = zc[q].x;
          r32[t0 + q] = rf[q];
        }
      }
      zm[0] = zc[0];
      zm[1] = zc[1];
      zc[0] = zp[0];
      zc[1] = zp[1];
    }
  }
  // per-block sums of r and r^2: float within a warp, FP64 across the warps
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int lane = (threadIdx.y * kSX + threadIdx.x) & 31, wid = (threadIdx.y * kSX + threadIdx.x) >> 5;
  if (lane == 0) {
    red[2 * wid] = (double)s1;
    red[2 * wid + 1] = (double)s2;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double d1 = 0.0, d2 = 0.0;
    for (int q = 0; q < kSX * kSY / 32; ++q) {
      d1 += red[2 * q];
      d2 += red[2 * q + 1];
    }
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * blk] = d1;
    partials[2 * blk + 1] = d2;
  }
}

// The same refinement pass with a native FP64 iterate (WGEO_PREC_FP64): the
// two iterate buffers hold doubles (8 bytes a cell, like a float-float pair),
// x_new = x + e and r = b - L x_new are formed on the FP64 pipe, and r, r^2
// are summed in FP64.  x32 = (float) x_new, r32 = (float) r.  A comparison
// point for the float-float pass above, which needs no FP64 arithmetic per
// cell.
__global__ void __launch_bounds__(kSX * kSY) update_residual_f64_kernel(PairD xp, const float* __restrict__ e,
                                                                        const float* __restrict__ b, int n,
                                                                        float* __restrict__ r32,
                                                                        float* __restrict__ x32,
                                                                        double* __restrict__ partials,
                                                                        SolveState* ss) {
  if (ss->done) return;
  __shared__ double red[2 * (kSX * kSY / 32)];
  const int cur = ss->xidx;
  const bool cold = ss->cold != 0;
  const double* __restrict__ xin = xp.buf[cur];
  double* __restrict__ xout = xp.buf[e ? cur ^ 1 : cur];
  const int I = blockIdx.x * kSX + threadIdx.x, j = blockIdx.y * kSY + threadIdx.y, k = blockIdx.z;
  const int i0 = 2 * I;
  const bool vec = (n & 1) == 0;
  double s1 = 0.0, s2 = 0.0;
  if (i0 < n && j < n) {
    const bool has1 = i0 + 1 < n;
    const int64_t nn = (int64_t)n * n;
    const int64_t t0 = (int64_t)k * nn + (int64_t)j * n + i0;
    auto one = [&](int64_t q) { return cold ? 0.0 : (e ? xin[q] + (double)e[q] : xin[q]); };
    auto pair = [&](int64_t q, double& a, double& c) {
      if (vec && !cold) {
        const double2 v = *reinterpret_cast<const double2*>(xin + q);
        a = v.x;
        c = v.y;
        if (e) {
          const float2 ev = *reinterpret_cast<const float2*>(e + q);
          a += (double)ev.x;
          c += (double)ev.y;
        }
      } else {
        a = one(q);
        c = has1 ? one(q + 1) : 0.0;
      }
    };
    double xc[2];
    pair(t0, xc[0], xc[1]);
    double acc[2] = {0.0, 0.0};
    if (!cold) {
      if (has1) {
        acc[0] += xc[1] - xc[0];
        acc[1] += xc[0] - xc[1];
      }
      if (i0 > 0) acc[0] += one(t0 - 1) - xc[0];
      if (i0 + 2 < n) acc[1] += one(t0 + 2) - xc[1];
      double a, c;
      if (j > 0) { pair(t0 - n, a, c); acc[0] += a - xc[0]; acc[1] += c - xc[1]; }
      if (j < n - 1) { pair(t0 + n, a, c); acc[0] += a - xc[0]; acc[1] += c - xc[1]; }
      if (k > 0) { pair(t0 - nn, a, c); acc[0] += a - xc[0]; acc[1] += c - xc[1]; }
      if (k < n - 1) { pair(t0 + nn, a, c); acc[0] += a - xc[0]; acc[1] += c - xc[1]; }
    }
    float rf[2] = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q == 1 && !has1) break;
      const double r = (double)b[t0 + q] - acc[q];
      rf[q] = (float)r;
      s1 += r;
      s2 += r * r;
    }
    if (vec) {
      if (e || cold) *reinterpret_cast<double2*>(xout + t0) = make_double2(xc[0], xc[1]);
      *reinterpret_cast<float2*>(x32 + t0) = make_float2((float)xc[0], (float)xc[1]);
      *reinterpret_cast<float2*>(r32 + t0) = make_float2(rf[0], rf[1]);
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q == 1 && !has1) break;
        if (e || cold) xout[t0 + q] = xc[q];
        x32[t0 + q] = (float)xc[q];
        r32[t0 + q] = rf[q];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int lane = (threadIdx.y * kSX + threadIdx.x) & 31, wid = (threadIdx.y * kSX + threadIdx.x) >> 5;
  if (lane == 0) {
    red[2 * wid] = s1;
    red[2 * wid + 1] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double d1 = 0.0, d2 = 0.0;
    for (int q = 0; q < kSX * kSY / 32; ++q) {
      d1 += red[2 * q];
      d2 += red[2 * q + 1];
    }
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * blk] = d1;
    partials[2 * blk + 1] = d2;
  }
}

// FP64 iterate <-> float-float pair, in place in the current buffer (the
// solve's index on the device): the surface stages, the adjoint and a warm
// start read the iterate as a float-float pair.
__global__ void ff_from_f64_kernel(PairD xp, const SolveState* __restrict__ ss, int64_t N) {
  double* x = xp.buf[ss->xidx];
  float2* f = reinterpret_cast<float2*>(x);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[t];
    const float hi = (float)v;
    f[t] = make_float2(hi, (float)(v - (double)hi));
  }
}
__global__ void f64_from_ff_kernel(PairD xp, const SolveState* __restrict__ ss, int64_t N) {
  double* x = xp.buf[ss->xidx];
  const float2* f = reinterpret_cast<const float2*>(x);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = f[t];
    x[t] = (double)v.x + (double)v.y;
  }
}

// ---------------------------------------------------------------- unlumped Galerkin operator
// The same refinement pass for L' (weights 2 on the 12 edge neighbours, 1 on
// the 8 corners, walls mirrored): the weighted neighbour differences are
// exact (doubling is exact) and summed by the same two-sum chain.  One x pair
// per thread, as update_residual_kernel, so the grid and the partials match.
__device__ __forceinline__ int q1_fold(int v, int n) { return min(max(v, 0), n - 1); }

template <typename TB>
__global__ void __launch_bounds__(kSX * kSY) update_residual_q1_kernel(PairFF xp, const float* __restrict__ e,
                                                                       const TB* __restrict__ b, int n,
                                                                       float* __restrict__ r32,
                                                                       float* __restrict__ x32,
                                                                       double* __restrict__ partials,
                                                                       SolveState* ss) {
  if (ss->done) return;
  __shared__ double red[2 * (kSX * kSY / 32)];
  const int cur = ss->xidx;
  const bool cold = ss->cold != 0;
  const float2* __restrict__ xin = xp.buf[cur];
  float2* __restrict__ xout = xp.buf[e ? cur ^ 1 : cur];
  const int I = blockIdx.x * kSX + threadIdx.x, j = blockIdx.y * kSY + threadIdx.y, k = blockIdx.z;
  float s1 = 0.f, s2 = 0.f;
  auto xnew = [&](int64_t q) {
    const float2 v = xin[q];
    return e ? ff_add_f(v, e[q]) : v;
  };
  for (int c = 0; c < 2; ++c) {
    const int i = 2 * I + c;
    if (i >= n || j >= n) break;
    const int64_t t = lin(i, j, k, n);
    float2 xc = make_float2(0.f, 0.f);
    float2 acc = make_float2(0.f, 0.f);
    if (!cold) {
      xc = xnew(t);
      float sh = 0.f, err = 0.f, lo = 0.f;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int nz = (dx != 0) + (dy != 0) + (dz != 0);
            if (nz < 2) continue;                       // the centre and the faces: weight 0
            const int qi = q1_fold(i + dx, n), qj = q1_fold(j + dy, n), qk = q1_fold(k + dz, n);
            if (qi == i && qj == j && qk == k) continue;   // folded onto the cell itself
            const float w = nz == 2 ? 2.f : 1.f;
            const float2 v = xnew(lin(qi, qj, qk, n));
            const float2 d = two_sum(v.x, -xc.x);
            const float2 q = two_sum(sh, w * d.x);
            sh = q.x;
            err = __fadd_rn(err, __fadd_rn(q.y, w * d.y));
            lo = __fadd_rn(lo, w * __fsub_rn(v.y, xc.y));
          }
      acc = two_sum(sh, __fadd_rn(err, lo));
    }
    float blo;
    const float bhi = rhs_hi(b, t, blo);
    const float2 r = ff_sub(make_float2(bhi, blo), acc);
    const float rf = r.x + r.y;
    s1 += rf;
    s2 += rf * rf;
    if (e || cold) xout[t] = xc;
    x32[t] = xc.x;
    r32[t] = rf;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int lane = (threadIdx.y * kSX + threadIdx.x) & 31, wid = (threadIdx.y * kSX + threadIdx.x) >> 5;
  if (lane == 0) {
    red[2 * wid] = (double)s1;
    red[2 * wid + 1] = (double)s2;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double d1 = 0.0, d2 = 0.0;
    for (int q = 0; q < kSX * kSY / 32; ++q) {
      d1 += red[2 * q];
      d2 += red[2 * q + 1];
    }
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * blk] = d1;
    partials[2 * blk + 1] = d2;
  }
}

// (L' x)_p and the weight sum of the neighbours that do not fold onto p
// (the diagonal of L' is minus that sum).
__device__ __forceinline__ float q1_apply(const float* __restrict__ x, int i, int j, int k, int n, float xc,
                                          float* wsum) {
  float acc = 0.f, ws = 0.f;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz < 2) continue;
        const int qi = q1_fold(i + dx, n), qj = q1_fold(j + dy, n), qk = q1_fold(k + dz, n);
        if (qi == i && qj == j && qk == k) continue;
        const float w = nz == 2 ? 2.f : 1.f;
        acc += w * (__ldg(x + lin(qi, qj, qk, n)) - xc);
        ws += w;
      }
  *wsum = ws;
  return acc;
}

constexpr float kQ1Omega = 8.f / 9.f;   // Jacobi damping: D^-1 A spans [3/4, 3/2] on the rough modes

// One damped Jacobi sweep on L' x = b - shift: xo = x + omega (L' x - (b - shift)) / W
// (W the folded weight sum; ZERO: x taken as 0).  One cell per thread.
template <bool ZERO>
__global__ void __launch_bounds__(kSX * kSY) jacobi_q1_kernel(const float* __restrict__ x, float* __restrict__ xo,
                                                              const float* __restrict__ b,
                                                              const float* __restrict__ shift, int n,
                                                              const int* __restrict__ gate) {
  if (*gate) return;
  const int i = blockIdx.x * kSX + threadIdx.x, j = blockIdx.y * kSY + threadIdx.y, k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int64_t t = lin(i, j, k, n);
  const float rhs = b[t] - (shift ? *shift : 0.f);
  if (ZERO) {
    float ws = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nz = (dx != 0) + (dy != 0) + (dz != 0);
          if (nz < 2) continue;
          const int qi = q1_fold(i + dx, n), qj = q1_fold(j + dy, n), qk = q1_fold(k + dz, n);
          if (qi == i && qj == j && qk == k) continue;
          ws += nz == 2 ? 2.f : 1.f;
        }
    xo[t] = ws > 0.f ? -kQ1Omega * rhs / ws : 0.f;
    return;
  }
  const float xc = x[t];
  float ws;
  const float lx = q1_apply(x, i, j, k, n, xc, &ws);
  xo[t] = ws > 0.f ? xc + kQ1Omega * (lx - rhs) / ws : xc;
}

// bc = 1/2 * sum over the 8 children of the residual b - shift - L' x.
__global__ void __launch_bounds__(kSX * kSY) restrict_q1_kernel(const float* __restrict__ x,
                                                                const float* __restrict__ b,
                                                                const float* __restrict__ shift, int n,
                                                                float* __restrict__ bc, const int* __restrict__ gate) {
  if (*gate) return;
  const int nc = n >> 1;
  const int I = blockIdx.x * kSX + threadIdx.x, J = blockIdx.y * kSY + threadIdx.y, K = blockIdx.z;
  if (I >= nc || J >= nc) return;
  const float sh = shift ? *shift : 0.f;
  float acc = 0.f;
  for (int ch = 0; ch < 8; ++ch) {
    const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
    const int64_t t = lin(i, j, k, n);
    float ws;
    const float lx = q1_apply(x, i, j, k, n, x[t], &ws);
    acc += (b[t] - sh) - lx;
  }
  bc[lin(I, J, K, nc)] = 0.5f * acc;
}

__global__ void residual32_kernel(const float* __restrict__ x, const float* __restrict__ b,
                                  const float* __restrict__ shift, int n,
                                  double* __restrict__ partials, const int* __restrict__ gate) {
  if (*gate) return;
  __shared__ float red[32];
  const int64_t N = (int64_t)n * n * n;
  const float sh = *shift;
  float s1 = 0.f, s2 = 0.f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
    const float xc = x[t];
    float acc = 0.f;
    if (i > 0) acc += x[t - 1] - xc;
    if (i < n - 1) acc += x[t + 1] - xc;
    if (j > 0) acc += x[t - n] - xc;
    if (j < n - 1) acc += x[t + n] - xc;
    if (k > 0) acc += x[t - (int64_t)n * n] - xc;
    if (k < n - 1) acc += x[t + (int64_t)n * n] - xc;
    const float r = (b[t] - sh) - acc;
    s1 += r;
    s2 += r * r;
  }
  s1 = warp_sumf(s1);
  s2 = warp_sumf(s2);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = s1;
  __syncthreads();
  float t1 = 0.f;
  if (threadIdx.x < 32) t1 = warp_sumf(l < kThreads / 32 ? red[l] : 0.f);
  __syncthreads();
  if (l == 0) red[w] = s2;
  __syncthreads();
  float t2 = 0.f;
  if (threadIdx.x < 32) t2 = warp_sumf(l < kThreads / 32 ? red[l] : 0.f);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = (double)t1;
    partials[2 * blockIdx.x + 1] = (double)t2;
  }
}

// Fixed-order reduction of the residual partials and the convergence test.
// fp32 != 0: sums in float (the plain FP32 comparator's dots).  flip != 0:
// this step wrote the corrected x64 into the other buffer.
// Kernels launched by the recorded solver loops' bodies (device-side loop: the
// body's launch count is added once per iteration that runs).
__device__ unsigned long long g_loop_launches;

// step >= 0: the step number and whether it is the last allowed come from the
// host (fixed launch sequence); step < 0: a recorded loop body, which counts
// from the device state.  cond != 0: set the loop's condition to "not done".
__global__ void finalize_kernel(const double* __restrict__ partials, int nblocks, int64_t N,
                                SolveState* ss, DevState* st, double tol, int step, int fp32, int flip,
                                cudaGraphConditionalHandle hc, int cond) {
  if (ss->done) return;
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  if (fp32) {
    if (threadIdx.x == 0) {
      float f1 = 0.f, f2 = 0.f;
      for (int i = 0; i < nblocks; ++i) {
        f1 += (float)partials[2 * i];
        f2 += (float)partials[2 * i + 1];
      }
      s1 = f1;
      s2 = f2;
    }
  } else {
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
      s1 += partials[2 * i];
      s2 += partials[2 * i + 1];
    }
    s1 = block_sum<1024>(s1, red);
    s2 = block_sum<1024>(s2, red);
  }
  if (threadIdx.x == 0) {
    if (step < 0) {
      step = ss->iter + 1;
      atomicAdd(&g_loop_launches, (unsigned long long)ss->body_launches);
    }
    const bool last = step >= ss->max_steps;
    if (flip) ss->xidx ^= 1;
    ss->cold = 0;
    const double mean = s1 / (double)N;
    const double rn = sqrt(fmax(s2 - s1 * mean, 0.0));
    ss->rmean = mean;
    ss->rmean32 = (float)mean;
    const double bn = ss->bnorm;
    const double rel = (bn > 0.0) ? rn / bn : 0.0;
    ss->rel = rel;
    ss->iter = step;
    if (bn <= 0.0 || (rel <= tol && step >= ss->min_steps)) {
      ss->done = 1;
    } else if (last) {
      atomicOr(&st->status, WGEO_STATUS_NOT_CONVERGED);
      ss->done = 1;
    }
    if (cond) cudaGraphSetConditional(hc, ss->done ? 0u : 1u);
  }
}
__global__ void solve_begin_kernel(SolveState* ss, int cold, int max_steps, int min_steps, int body_launches) {
  ss->done = 0;
  ss->iter = 0;
  ss->rel = 0.0;
  ss->rmean = 0.0;
  ss->rmean32 = 0.f;
  ss->cold = cold;
  ss->max_steps = max_steps;
  ss->min_steps = min(min_steps, max_steps);
  ss->body_launches = body_launches;
}

// ---------------------------------------------------------------- levels above 16^3
// Plain kernels, one launch per step, each close to its memory floor.  A
// red-black half-sweep reads only cells of the other colour, so its updates
// are independent: a thread owns one x pair of cells (one of each colour)
// and updates the one of the sweep's colour in place.  x is read once from
// HBM per half-sweep (neighbour reuse through L1/L2), b and the written half
// once: about 8 bytes per cell.  Grids are 3D (32 pairs x 8 rows per block,
// one z plane per blockIdx.z), so no thread divides to find its cell.

__device__ __forceinline__ float prolong_at(const float* __restrict__ xc, int nc, int gx, int gy, int gz) {
  const int I = gx >> 1, J = gy >> 1, K = gz >> 1;
  const int I2 = min(max((gx & 1) ? I + 1 : I - 1, 0), nc - 1);
  const int J2 = min(max((gy & 1) ? J + 1 : J - 1, 0), nc - 1);
  const int K2 = min(max((gz & 1) ? K + 1 : K - 1, 0), nc - 1);
  const float a = 0.75f, c = 0.25f;
  return a * a * a * xc[lin(I, J, K, nc)] + c * a * a * xc[lin(I2, J, K, nc)] +
         a * c * a * xc[lin(I, J2, K, nc)] + a * a * c * xc[lin(I, J, K2, nc)] +
         c * c * a * xc[lin(I2, J2, K, nc)] + c * a * c * xc[lin(I2, J, K2, nc)] +
         a * c * c * xc[lin(I, J2, K2, nc)] + c * c * c * xc[lin(I2, J2, K2, nc)];
}

// One half-sweep of colour `color` ((i + j + k) & 1 == color) on
// L x = b - shift.  ZERO: x is taken as 0 (the first half-sweep of a cycle
// from a zero start), and the pair's other cell is written 0.
template <bool ZERO>
__global__ void __launch_bounds__(kSX * kSY) rb_half_kernel(float* __restrict__ x, const float* __restrict__ b,
                                                            const float* __restrict__ shift, int n, int color,
                                                            const int* __restrict__ gate) {
  if (*gate) return;
  const int ih = blockIdx.x * kSX + threadIdx.x, j = blockIdx.y * kSY + threadIdx.y, k = blockIdx.z;
  if (2 * ih >= n || j >= n) return;
  const float sh = shift ? *shift : 0.f;
  const int odd = (j + k + color) & 1;
  const int i = 2 * ih + odd;
  const int64_t nn = (int64_t)n * n;
  const int64_t p = k * nn + (int64_t)j * n + i;
  const int cnt = 6 - (i == 0) - (i == n - 1) - (j == 0) - (j == n - 1) - (k == 0) - (k == n - 1);
  float acc = 0.f;
  if (!ZERO) {
    if (i > 0) acc += x[p - 1];
    if (i < n - 1) acc += x[p + 1];
    if (j > 0) acc += x[p - n];
    if (j < n - 1) acc += x[p + n];
    if (k > 0) acc += x[p - nn];
    if (k < n - 1) acc += x[p + nn];
  }
  x[p] = __fdividef(acc - (__ldg(b + p) - sh), (float)cnt);
  if (ZERO) x[p + (odd ? -1 : 1)] = 0.f;
}

// bc = 1/2 * sum over the 8 children of the residual b - shift - L x.
__global__ void __launch_bounds__(kSX * kSY) restrict_kernel(const float* __restrict__ x,
                                                             const float* __restrict__ b,
                                                             const float* __restrict__ shift, int n,
                                                             float* __restrict__ bc,
                                                             const int* __restrict__ gate) {
  if (*gate) return;
  const int nc = n >> 1;
  const int I = blockIdx.x * kSX + threadIdx.x, J = blockIdx.y * kSY + threadIdx.y, K = blockIdx.z;
  if (I >= nc || J >= nc) return;
  const float sh = shift ? *shift : 0.f;
  const int64_t nn = (int64_t)n * n;
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    const int64_t p = k * nn + (int64_t)j * n + i;
    const float xv = x[p];
    float lx = 0.f;
    if (i > 0) lx += x[p - 1] - xv;
    if (i < n - 1) lx += x[p + 1] - xv;
    if (j > 0) lx += x[p - n] - xv;
    if (j < n - 1) lx += x[p + n] - xv;
    if (k > 0) lx += x[p - nn] - xv;
    if (k < n - 1) lx += x[p + nn] - xv;
    acc += (__ldg(b + p) - sh) - lx;
  }
  bc[((int64_t)K * nc + J) * nc + I] = 0.5f * acc;
}

// x += P xc for one x pair (2I, 2I+1) of row j, plane k: trilinear weights
// 3/4, 1/4 per axis toward the nearer coarse neighbour (mirrored at the
// walls), from the 12 coarse values the pair needs.
__global__ void __launch_bounds__(kSX * kSY) prolong_pair_kernel(const float* __restrict__ xc,
                                                                 float* __restrict__ x, int n,
                                                                 const int* __restrict__ gate) {
  if (*gate) return;
  const int nc = n >> 1;
  const int I = blockIdx.x * kSX + threadIdx.x, j = blockIdx.y * kSY + threadIdx.y, k = blockIdx.z;
  if (I >= nc || j >= n) return;
  const int J = j >> 1, K = k >> 1;
  const int J2 = min(max((j & 1) ? J + 1 : J - 1, 0), nc - 1);
  const int K2 = min(max((k & 1) ? K + 1 : K - 1, 0), nc - 1);
  const int Im = max(I - 1, 0), Ip = min(I + 1, nc - 1);
  const int64_t ncc = (int64_t)nc * nc;
  const int64_t r[4] = {K * ncc + (int64_t)J * nc, K * ncc + (int64_t)J2 * nc, K2 * ncc + (int64_t)J * nc,
                        K2 * ncc + (int64_t)J2 * nc};
  const float w[4] = {0.5625f, 0.1875f, 0.1875f, 0.0625f};
  float ve = 0.f, vo = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float a0 = __ldg(xc + r[q] + I), am = __ldg(xc + r[q] + Im), ap = __ldg(xc + r[q] + Ip);
    ve += w[q] * (0.75f * a0 + 0.25f * am);
    vo += w[q] * (0.75f * a0 + 0.25f * ap);
  }
  float2* xp = reinterpret_cast<float2*>(x + (int64_t)k * n * n + (int64_t)j * n + 2 * I);
  float2 v = *xp;
  v.x += ve;
  v.y += vo;
  *xp = v;
}

// ---------------------------------------------------------------- small grids
// A whole V-cycle hierarchy for n <= 16 in one CTA's shared memory: solves
// L x = b - shift - mean approximately, writes x.  With a hierarchy above a
// coarsest level of at most 4^3: one V-cycle from zero, 2n + 8 red-black
// sweeps on the coarsest level; as the coarse-grid correction of the outer
// cycle it needs no more (on the 256^3 benchmark the refinement takes the
// same number of steps as with two cycles and 2n^2 + 16 sweeps).  Otherwise
// (a single level, e.g. an odd grid, or a larger coarsest level): two
// V-cycles, 2n^2 + 16 sweeps on the coarsest level.
constexpr int kSmallCap = 4096 + 512 + 64 + 27 + 8;
constexpr int kSmallCycles = 1;     // V-cycles of the coarse-grid solve

__device__ void small_rbgs(float* x, const float* b, int n, int color) {
  const int N = n * n * n;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int i = t % n, j = (t / n) % n, k = t / (n * n);
    if (((i + j + k) & 1) != color) continue;
    float acc = 0.f;
    int cnt = 0;
    if (i > 0) { acc += x[t - 1]; ++cnt; }
    if (i < n - 1) { acc += x[t + 1]; ++cnt; }
    if (j > 0) { acc += x[t - n]; ++cnt; }
    if (j < n - 1) { acc += x[t + n]; ++cnt; }
    if (k > 0) { acc += x[t - n * n]; ++cnt; }
    if (k < n - 1) { acc += x[t + n * n]; ++cnt; }
    x[t] = cnt ? (acc - b[t]) / (float)cnt : 0.f;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) small_vcycle_kernel(float* __restrict__ xg, const float* __restrict__ bg,
                                                            const float* __restrict__ shift, int n0,
                                                            const int* __restrict__ gate) {
  if (*gate) return;
  __shared__ float xs[kSmallCap];
  __shared__ float bsm[kSmallCap];
  __shared__ double red[32];
  __shared__ float meanb;
  int ns[8], off[8], L = 0;
  {
    int n = n0, o = 0;
    while (true) {
      ns[L] = n;
      off[L] = o;
      o += n * n * n;
      ++L;
      if ((n % 2) != 0 || n <= 4 || L == 8) break;
      n /= 2;
    }
  }
  const int N0 = n0 * n0 * n0;
  const float sh = shift ? *shift : 0.f;
  double s = 0.0;
  for (int t = threadIdx.x; t < N0; t += blockDim.x) {
    const float v = bg[t] - sh;
    bsm[t] = v;
    xs[t] = 0.f;
    s += v;
  }
  s = block_sum<1024>(s, red);
  if (threadIdx.x == 0) meanb = (float)(s / N0);
  __syncthreads();
  for (int t = threadIdx.x; t < N0; t += blockDim.x) bsm[t] -= meanb;
  __syncthreads();
  const int cycles = L > 1 ? kSmallCycles : 2;
  for (int cyc = 0; cyc < cycles; ++cyc) {
    // down
    for (int l = 0; l < L - 1; ++l) {
      const int n = ns[l];
      float* x = xs + off[l];
      const float* b = bsm + off[l];
      for (int sw = 0; sw < kNu; ++sw) {
        small_rbgs(x, b, n, 0);
        small_rbgs(x, b, n, 1);
      }
      const int nc = ns[l + 1];
      float* xcn = xs + off[l + 1];
      float* bcn = bsm + off[l + 1];
      for (int t = threadIdx.x; t < nc * nc * nc; t += blockDim.x) {
        const int I = t % nc, J = (t / nc) % nc, K = t / (nc * nc);
        float acc = 0.f;
        for (int ch = 0; ch < 8; ++ch) {
          const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
          const int p = (k * n + j) * n + i;
          const float xv = x[p];
          float lx = 0.f;
          if (i > 0) lx += x[p - 1] - xv;
          if (i < n - 1) lx += x[p + 1] - xv;
          if (j > 0) lx += x[p - n] - xv;
          if (j < n - 1) lx += x[p + n] - xv;
          if (k > 0) lx += x[p - n * n] - xv;
          if (k < n - 1) lx += x[p + n * n] - xv;
          acc += b[p] - lx;
        }
        bcn[t] = 0.5f * acc;
        xcn[t] = 0.f;
      }
      __syncthreads();
    }
    // coarsest
    {
      const int n = ns[L - 1];
      float* x = xs + off[L - 1];
      const float* b = bsm + off[L - 1];
      // a coarsest level of at most 4^3 below a hierarchy needs only a rough
      // solve; a larger one (no hierarchy, e.g. an odd grid) is the whole solve
      const int sweeps = (n <= 4 && L > 1) ? 2 * n + 8 : 2 * n * n + 16;
      for (int sw = 0; sw < sweeps; ++sw) {
        small_rbgs(x, b, n, 0);
        small_rbgs(x, b, n, 1);
      }
    }
    // up
    for (int l = L - 2; l >= 0; --l) {
      const int n = ns[l], nc = ns[l + 1];
      float* x = xs + off[l];
      const float* b = bsm + off[l];
      const float* xcn = xs + off[l + 1];
      for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, k = t / (n * n);
        x[t] += prolong_at(xcn, nc, i, j, k);
      }
      __syncthreads();
      for (int sw = 0; sw < kNu; ++sw) {
        small_rbgs(x, b, n, 1);
        small_rbgs(x, b, n, 0);
      }
    }
  }
  for (int t = threadIdx.x; t < N0; t += blockDim.x) xg[t] = xs[t];
}

// The same hierarchy for L' with Gauss-Seidel in 8 colours ((i, j, k) mod 2:
// no two cells of a colour are neighbours in the 27-point stencil), in place.
__device__ void small_gs8(float* x, const float* b, int n, int color) {
  const int N = n * n * n;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int i = t % n, j = (t / n) % n, k = t / (n * n);
    if (((i & 1) | ((j & 1) << 1) | ((k & 1) << 2)) != color) continue;
    float acc = 0.f, ws = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nz = (dx != 0) + (dy != 0) + (dz != 0);
          if (nz < 2) continue;
          const int qi = q1_fold(i + dx, n), qj = q1_fold(j + dy, n), qk = q1_fold(k + dz, n);
          if (qi == i && qj == j && qk == k) continue;
          const float w = nz == 2 ? 2.f : 1.f;
          acc += w * x[(qk * n + qj) * n + qi];
          ws += w;
        }
    x[t] = ws > 0.f ? (acc - b[t]) / ws : 0.f;
  }
  __syncthreads();
}

__device__ float small_q1_residual(const float* x, const float* b, int n, int i, int j, int k) {
  const int p = (k * n + j) * n + i;
  const float xv = x[p];
  float lx = 0.f;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz < 2) continue;
        const int qi = q1_fold(i + dx, n), qj = q1_fold(j + dy, n), qk = q1_fold(k + dz, n);
        if (qi == i && qj == j && qk == k) continue;
        lx += (nz == 2 ? 2.f : 1.f) * (x[(qk * n + qj) * n + qi] - xv);
      }
  return b[p] - lx;
}

__global__ void __launch_bounds__(1024) small_vcycle_q1_kernel(float* __restrict__ xg, const float* __restrict__ bg,
                                                               const float* __restrict__ shift, int n0,
                                                               const int* __restrict__ gate) {
  if (*gate) return;
  __shared__ float xs[kSmallCap];
  __shared__ float bsm[kSmallCap];
  __shared__ double red[32];
  __shared__ float meanb;
  int ns[8], off[8], L = 0;
  {
    int n = n0, o = 0;
    while (true) {
      ns[L] = n;
      off[L] = o;
      o += n * n * n;
      ++L;
      if ((n % 2) != 0 || n <= 4 || L == 8) break;
      n /= 2;
    }
  }
  const int N0 = n0 * n0 * n0;
  const float sh = shift ? *shift : 0.f;
  double s = 0.0;
  for (int t = threadIdx.x; t < N0; t += blockDim.x) {
    const float v = bg[t] - sh;
    bsm[t] = v;
    xs[t] = 0.f;
    s += v;
  }
  s = block_sum<1024>(s, red);
  if (threadIdx.x == 0) meanb = (float)(s / N0);
  __syncthreads();
  for (int t = threadIdx.x; t < N0; t += blockDim.x) bsm[t] -= meanb;
  __syncthreads();
  const int cycles = L > 1 ? kSmallCycles : 2;
  for (int cyc = 0; cyc < cycles; ++cyc) {
    for (int l = 0; l < L - 1; ++l) {
      const int n = ns[l];
      float* x = xs + off[l];
      const float* b = bsm + off[l];
      for (int sw = 0; sw < kNu; ++sw)
        for (int c = 0; c < 8; ++c) small_gs8(x, b, n, c);
      const int nc = ns[l + 1];
      float* xcn = xs + off[l + 1];
      float* bcn = bsm + off[l + 1];
      for (int t = threadIdx.x; t < nc * nc * nc; t += blockDim.x) {
        const int I = t % nc, J = (t / nc) % nc, K = t / (nc * nc);
        float acc = 0.f;
        for (int ch = 0; ch < 8; ++ch)
          acc += small_q1_residual(x, b, n, 2 * I + (ch & 1), 2 * J + ((ch >> 1) & 1), 2 * K + (ch >> 2));
        bcn[t] = 0.5f * acc;
        xcn[t] = 0.f;
      }
      __syncthreads();
    }
    {
      const int n = ns[L - 1];
      float* x = xs + off[L - 1];
      const float* b = bsm + off[L - 1];
      const int sweeps = (n <= 4 && L > 1) ? 2 * n + 8 : 2 * n * n + 16;
      for (int sw = 0; sw < sweeps; ++sw)
        for (int c = 0; c < 8; ++c) small_gs8(x, b, n, c);
    }
    for (int l = L - 2; l >= 0; --l) {
      const int n = ns[l], nc = ns[l + 1];
      float* x = xs + off[l];
      const float* b = bsm + off[l];
      const float* xcn = xs + off[l + 1];
      for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, k = t / (n * n);
        x[t] += prolong_at(xcn, nc, i, j, k);
      }
      __syncthreads();
      for (int sw = 0; sw < kNu; ++sw)
        for (int c = 7; c >= 0; --c) small_gs8(x, b, n, c);
    }
  }
  for (int t = threadIdx.x; t < N0; t += blockDim.x) xg[t] = xs[t];
}

// dchi *= s (the adjoint right-hand side of the scaled operator L' = 12 L).
__global__ void scale64_kernel(double* __restrict__ v, int64_t N, double s) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x)
    v[t] *= s;
}

// out32 (may be null): b rounded to float, the first residual of a solve
// from zero (its head skipped).
__global__ void rhs_stats64_kernel(const double* __restrict__ b, int64_t N,
                                   double* __restrict__ partials, float* __restrict__ out32) {
  __shared__ double red[32];
  // per thread: the sum in float-float, the sum of squares in float (it only
  // sets the tolerance's scale); FP64 from the block sums on
  float2 f1 = make_float2(0.f, 0.f);
  float f2 = 0.f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = split_f64(b[t]);
    f1 = ff_add_f(ff_add_f(f1, v.x), v.y);
    f2 = fmaf(v.x, v.x, f2);
    if (out32) out32[t] = __fadd_rn(v.x, v.y);
  }
  double s1 = (double)f1.x + (double)f1.y, s2 = (double)f2;
  s1 = block_sum<kThreads>(s1, red);
  s2 = block_sum<kThreads>(s2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1;
    partials[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void rhs_stats_finalize_kernel(const double* __restrict__ partials, int nblocks,
                                          int64_t N, SolveState* ss) {
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    s1 += partials[2 * i];
    s2 += partials[2 * i + 1];
  }
  s1 = block_sum<1024>(s1, red);
  s2 = block_sum<1024>(s2, red);
  if (threadIdx.x == 0) {
    const double mean = s1 / (double)N;
    ss->bmean = mean;
    ss->bmean32 = (float)mean;
    ss->bnorm = sqrt(fmax(s2 - s1 * mean, 0.0));
  }
}

// One V-cycle on level l, in place.  x0: level-0 iterate; b0, shift0:
// level-0 right-hand side.  zero0: level-0 x starts at zero.
int vcycle_q1(wgeo_handle* h, int l, float* x0, const float* b0, const float* shift0, bool zero0, float* t0,
              const int* gate, cudaStream_t s);

int vcycle(wgeo_handle* h, int l, float* x0, const float* b0, const float* shift0, bool zero0,
           const int* gate, cudaStream_t s) {
  const int n = h->levels[l].n;
  float* x = (l == 0) ? x0 : h->levels[l].x;
  const float* b = (l == 0) ? b0 : h->levels[l].b;
  const float* shift = (l == 0) ? shift0 : nullptr;
  if (n <= kSmallN || l == h->nlevels - 1) {
    small_vcycle_kernel<<<1, 1024, 0, s>>>(x, b, shift, n, gate);
    WGEO_LAUNCH_CHECK();
    return WGEO_OK;
  }
  const bool zero = (l == 0) ? zero0 : true;
  const int nc = n >> 1;
  const dim3 blk(kSX, kSY);
  const dim3 gf(div_up(nc, kSX), div_up(n, kSY), n);      // fine pairs
  const dim3 gc(div_up(nc, kSX), div_up(nc, kSY), nc);    // coarse cells
  // pre-smoothing: kNu red-black sweeps, red first (the first from zero when zero)
  for (int sw = 0; sw < kNu; ++sw)
    for (int c = 0; c < 2; ++c) {
      if (zero && sw == 0 && c == 0)
        rb_half_kernel<true><<<gf, blk, 0, s>>>(x, b, shift, n, c, gate);
      else
        rb_half_kernel<false><<<gf, blk, 0, s>>>(x, b, shift, n, c, gate);
      WGEO_LAUNCH_CHECK();
    }
  restrict_kernel<<<gc, blk, 0, s>>>(x, b, shift, n, h->levels[l + 1].b, gate);
  WGEO_LAUNCH_CHECK();
  int rc = vcycle(h, l + 1, x0, b0, shift0, zero0, gate, s);
  if (rc) return rc;
  prolong_pair_kernel<<<gf, blk, 0, s>>>(h->levels[l + 1].x, x, n, gate);
  WGEO_LAUNCH_CHECK();
  // post-smoothing: kNu sweeps, black first
  for (int sw = 0; sw < kNu; ++sw)
    for (int c = 1; c >= 0; --c) {
      rb_half_kernel<false><<<gf, blk, 0, s>>>(x, b, shift, n, c, gate);
      WGEO_LAUNCH_CHECK();
    }
  return WGEO_OK;
}

// ---------------------------------------------------------------- spectral correction
// With the walls mirrored, both operators are diagonal in the cosine basis
// c_k(i) = cos(pi k (i + 1/2) / n) per axis: the 7-point L has eigenvalue
// -(s_x + s_y + s_z), s = 4 sin^2(pi k / 2n), and the scaled Galerkin L' has
// -12 (s_x m_y m_z + m_x s_y m_z + m_x m_y s_z), m = 1 - s / 6.  So a
// correction L e = r - mean(r) is solved directly: the (unnormalised)
// DCT-II along x, y and z, a division by the eigenvalue (the zero mode, the
// mean, dropped), and the exact inverse transform along z, y and x.  Five
// in-place passes over the grid (the z pass divides and transforms back).
//
// Each one-dimensional DCT-II of n points goes through an n-point complex FFT
// (Makhoul, IEEE TASSP 1980): v_m = x_{2m}, v_{n-1-m} = x_{2m+1}, X_k =
// Re(e^{-i pi k / 2n} V_k).  Its inverse: V_k = e^{i pi k / 2n} (X_k - i
// X_{n-k}) (X_n = 0), v = IFFT(V) = conj(FFT(conj V)) / n.  Two real lines
// share one complex FFT (Z = v_a + i v_b; V_a, V_b from Z_k and conj Z_{n-k};
// back, IFFT(V_a + i V_b) = v_a + i v_b), one warp per pair.
//
// The FFT of n = 32 R points in a warp (the four-step split n = R x 32): lane
// j holds z_{j + 32 m} in register m; an R-point DFT over m in registers, the
// twiddle e^{-2 pi i j a / n}, and a 32-point DFT across the lanes by xor
// shuffles (decimation in frequency), after which lane j register a holds
// Z_{a + R brev5(j)}.  The transposed sequence (decimation in time across the
// lanes, twiddle, register DFT) takes that layout back to j + 32 m, so the z
// pass never leaves registers.  Shared memory holds the block's 32 lines
// (padded rows: the coalesced tile copies and the scattered lane accesses are
// both free of bank conflicts) and the twiddle tables; power-of-two
// 32 <= n <= 512.
constexpr int kDctTile = 32;      // lines per block: 16 warps, two lines each
constexpr int kDctThreads = 512;
constexpr unsigned kFull = 0xffffffffu;

bool use_spectral(const wgeo_handle* h, int n) {
  return h->opt.spectral && n >= 32 && n <= 512 && (n & (n - 1)) == 0;
}

__host__ __device__ constexpr int dct_ls(int n) { return (n + n / 32) | 1; }   // odd row stride
__device__ __forceinline__ int dct_at(int i) { return i + (i >> 5); }
// Compiler-only fence between the FFT phases: the shared twiddle tables are
// read again after it instead of being held in registers across phases.
__device__ __forceinline__ void phase_fence() { asm volatile("" ::: "memory"); }
__device__ __forceinline__ int brev5(int j) { return (int)(__brev((unsigned)j) >> 27); }

template <int R>
constexpr size_t dct_smem() {
  return sizeof(float2) * (32 * R + 160 + 32 * R + 16) + sizeof(float) * 32 * R +
         sizeof(float) * kDctTile * dct_ls(32 * R);
}

__global__ void dct_tables_kernel(int n, float2* __restrict__ t1, float2* __restrict__ w32,
                                  float2* __restrict__ wml, float2* __restrict__ tr,
                                  float* __restrict__ sk, float* __restrict__ skl,
                                  float2* __restrict__ tw, float2* __restrict__ wq) {
  const int R = n / 32;
  const int count = n > 160 ? n + 1 : 161;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    double sn, cs;
    if (q <= n) {
      sincospi((double)q / (2.0 * n), &sn, &cs);
      wq[q] = make_float2((float)cs, (float)-sn);   // e^{-i pi q / (2 n)}
    }
    if (q < n) {
      sincospi(2.0 * (double)q / n, &sn, &cs);
      tw[q] = make_float2((float)cs, (float)-sn);   // e^{-2 pi i q / n}
    }
    const int a = q >> 5, j = q & 31;
    if (q < n) {
      sincospi(2.0 * (double)(j * a) / n, &sn, &cs);
      t1[q] = make_float2((float)cs, (float)-sn);
      const int k = a + R * (int)(__brev((unsigned)j) >> 27);
      sincospi((double)k / (2.0 * n), &sn, &cs);
      wml[q] = make_float2((float)cs, (float)-sn);
      skl[q] = (float)(4.0 * sn * sn);
      sincospi((double)q / (2.0 * n), &sn, &cs);
      sk[q] = (float)(4.0 * sn * sn);
    }
    if (q < 160) {
      // stage a combines pairs of hh-point DFTs; only the upper lane of a
      // pair (j & hh) multiplies, the lower one holds 1 so that both run the
      // same instructions
      const int hh = 1 << a;
      sincospi((double)(j & (hh - 1)) / hh, &sn, &cs);
      w32[q] = (j & hh) ? make_float2((float)cs, (float)-sn) : make_float2(1.f, 0.f);
    }
    if (q < R) {
      sincospi(2.0 * q / R, &sn, &cs);
      tr[q] = make_float2((float)cs, (float)-sn);
    }
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}

template <int R>
__host__ __device__ constexpr int rev_bits(int k) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((k & b) ? 1 : 0);
  return r;
}

// v <- DFT_R(v) (e^{-2 pi i q a / R}), natural order in and out: radix-2
// decimation in frequency, then the bit reversal as a register renaming.
template <int R>
__device__ __forceinline__ void dft_regs(float2 (&v)[R], const float2* tr) {
#pragma unroll
  for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
    for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
      for (int t = 0; t < h; ++t) {
        const float2 x = v[g + t], y = v[g + t + h];
        v[g + t] = cadd(x, y);
        v[g + t + h] = t == 0 ? csub(x, y) : cmul(csub(x, y), tr[t * (R / (2 * h))]);
      }
    }
  }
  float2 w[R];
#pragma unroll
  for (int k = 0; k < R; ++k) w[k] = v[rev_bits<R>(k)];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = w[k];
}

// Forward FFT of the warp's line: in, lane j register m = z_{j + 32 m}; out,
// lane j register a = Z_{a + R brev5(j)}.
template <int R>
__device__ __forceinline__ void fft_warp_dif(float2 (&v)[R], const float2* t1, const float2* w32,
                                             const float2* tr, int lane) {
  dft_regs<R>(v, tr);
#pragma unroll
  for (int a = 1; a < R; ++a) v[a] = cmul(v[a], t1[a * 32 + lane]);
#pragma unroll
  for (int st = 4; st >= 0; --st) {
    const int h = 1 << st;
    // upper lane: (p - v) w; lower lane: (v + p) 1 (its table entry)
    const float sg = (lane & h) ? -1.f : 1.f;
    const float2 w = w32[st * 32 + lane];
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const float2 p = shfl_xor2(v[a], h);
      v[a] = cmul(make_float2(fmaf(sg, v[a].x, p.x), fmaf(sg, v[a].y, p.y)), w);
    }
  }
}

// Forward FFT with the layouts swapped: in, lane j register a = u_{a + R
// brev5(j)}; out, lane j register m = U_{j + 32 m}.
template <int R>
__device__ __forceinline__ void fft_warp_dit(float2 (&v)[R], const float2* t1, const float2* w32,
                                             const float2* tr, int lane) {
#pragma unroll
  for (int st = 0; st <= 4; ++st) {
    const int h = 1 << st;
    // upper lane: p - v w; lower lane: v 1 + p (its table entry is 1)
    const float sg = (lane & h) ? -1.f : 1.f;
    const float2 w = w32[st * 32 + lane];
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const float2 m = cmul(v[a], w);
      const float2 p = shfl_xor2(m, h);
      v[a] = make_float2(fmaf(sg, m.x, p.x), fmaf(sg, m.y, p.y));
    }
  }
#pragma unroll
  for (int a = 1; a < R; ++a) v[a] = cmul(v[a], t1[a * 32 + lane]);
  dft_regs<R>(v, tr);
}

// v[a] <- f(a, v[a], c_a) for every register, c_a the value at index n - k
// of the layout k = a + R brev5(lane) (index 0 maps to itself, or to zero
// with ZERO_ORIGIN); the registers are taken in mirrored pairs (a, R - a), so
// that only a pair's partners are live at a time.
template <int R, bool ZERO_ORIGIN, class F>
__device__ __forceinline__ void mirror_apply(float2 (&v)[R], int lane, F f) {
  float2 c0 = shfl2(v[0], brev5((32 - brev5(lane)) & 31));
  if (ZERO_ORIGIN && lane == 0) c0 = make_float2(0.f, 0.f);
  if (R > 1) {
    const float2 ch = shfl_xor2(v[R / 2], 31);
#pragma unroll
    for (int a = 1; a < R / 2; ++a) {
      const float2 ca = shfl_xor2(v[R - a], 31), cb = shfl_xor2(v[a], 31);
      v[a] = f(a, v[a], ca);
      v[R - a] = f(R - a, v[R - a], cb);
    }
    v[R / 2] = f(R / 2, v[R / 2], ch);
  }
  v[0] = f(0, v[0], c0);
}

// The conjugate of the packed inverse input: for each line conj(V_k) =
// e^{-i pi k/2n} (X_k + i X_{n-k}), and conj(V_a + i V_b) = conj V_a - i conj V_b.
__device__ __forceinline__ float2 inverse_input(float2 w, float xa, float xan, float xb, float xbn) {
  const float2 ca = cmul(w, make_float2(xa, xan)), cb = cmul(w, make_float2(xb, xbn));
  return make_float2(ca.x + cb.y, ca.y - cb.x);
}

// Position of v_p in x: v_p = x_{2p} (p < n/2), x_{2(n-1-p)+1} (p >= n/2).
__device__ __forceinline__ int dct_src(int p, int n) { return p < (n >> 1) ? 2 * p : 2 * (n - 1 - p) + 1; }

// MODE 0: forward DCT-II along `axis`; 1: its inverse; 2 (axis z): forward,
// division by the eigenvalue, inverse.  A block takes 32 lines: along x, 32
// rows of one plane; along y or z, 32 neighbouring x columns.  `in` may be `out`
// (each block reads and writes only its own lines).
template <int R, int MODE>
__global__ void __launch_bounds__(kDctThreads, R <= 8 ? 2 : 1)
    dct_pass_kernel(const float* in, float* out, int axis, const float2* __restrict__ t1g,
                    const float2* __restrict__ w32g, const float2* __restrict__ wmg,
                    const float2* __restrict__ trg, const float* __restrict__ skg,
                    const float* __restrict__ sklg, int q1, const int* __restrict__ gate) {
  constexpr int n = 32 * R;
  constexpr int LS = dct_ls(n);
  constexpr int kVec = kDctTile * n / 4;                       // float4 per tile
  constexpr int kIt = (kVec + kDctThreads - 1) / kDctThreads;
  if (*gate) return;
  extern __shared__ float4 dsm4[];
  float2* t1 = reinterpret_cast<float2*>(dsm4);
  float2* w32 = t1 + n;
  float2* wm = w32 + 160;
  float2* tr = wm + n;
  float* skl = reinterpret_cast<float*>(tr + 16);
  float* S = skl + n;
  const int tid = threadIdx.x;
  for (int q = tid; q < n; q += kDctThreads) {
    t1[q] = t1g[q];
    wm[q] = wmg[q];
    if (MODE == 2) skl[q] = sklg[q];
  }
  if (tid < 160) w32[tid] = w32g[tid];
  if (tid < R) tr[tid] = trg[tid];

  const int groups = n / kDctTile;
  const int fixed = blockIdx.x / groups, t0 = (blockIdx.x - fixed * groups) * kDctTile;
  // tile element (l, i) -> grid; along x the tile is 32 n contiguous floats,
  // along y or z n rows of 32 contiguous floats
  const int64_t nn = (int64_t)n * n;
  const int64_t base = axis == 0 ? ((int64_t)fixed * n + t0) * n : axis == 1 ? fixed * nn + t0 : (int64_t)fixed * n + t0;
  const int64_t rstride = axis == 1 ? n : nn;
  {
    float4 buf[kIt];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kDctThreads;
      if (q < kVec) {
        const int64_t g = axis == 0 ? base + 4 * (int64_t)q : base + (q >> 3) * rstride + 4 * (q & 7);
        buf[it] = *reinterpret_cast<const float4*>(in + g);
      }
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kDctThreads;
      if (q < kVec) {
        const float e[4] = {buf[it].x, buf[it].y, buf[it].z, buf[it].w};
        if (axis == 0) {
          const int l = (4 * q) / n, i = (4 * q) % n;
#pragma unroll
          for (int c = 0; c < 4; ++c) S[l * LS + dct_at(i + c)] = e[c];
        } else {
          const int i = q >> 3, l = 4 * (q & 7);
#pragma unroll
          for (int c = 0; c < 4; ++c) S[(l + c) * LS + dct_at(i)] = e[c];
        }
      }
    }
  }
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  float* Sa = S + (2 * warp) * LS;
  float* Sb = Sa + LS;
  const int bl = brev5(lane);
  float2 v[R];
  if (MODE == 1) {
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const int k = a + R * bl;
      const float xa = Sa[dct_at(k)], xb = Sb[dct_at(k)];
      const float xan = k ? Sa[dct_at(n - k)] : 0.f, xbn = k ? Sb[dct_at(n - k)] : 0.f;
      v[a] = inverse_input(wm[a * 32 + lane], xa, xan, xb, xbn);
    }
  } else {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int s = dct_at(dct_src(lane + 32 * m, n));
      v[m] = make_float2(Sa[s], Sb[s]);
    }
    fft_warp_dif<R>(v, t1, w32, tr, lane);
    phase_fence();
    // X_k of both lines: V_a = (Z_k + conj Z_{n-k}) / 2, V_b = (Z_k - conj Z_{n-k}) / 2i
    mirror_apply<R, false>(v, lane, [&](int a, float2 z, float2 c) {
      const float2 va = make_float2(0.5f * (z.x + c.x), 0.5f * (z.y - c.y));
      const float2 vb = make_float2(0.5f * (z.y + c.y), 0.5f * (c.x - z.x));
      const float2 w = wm[a * 32 + lane];
      return make_float2(w.x * va.x - w.y * va.y, w.x * vb.x - w.y * vb.y);
    });
    phase_fence();
    if (MODE == 0) {
      __syncwarp();
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const int s = dct_at(a + R * bl);
        Sa[s] = v[a].x;
        Sb[s] = v[a].y;
      }
    } else {
      // divide by the eigenvalue of mode (kx, ky, kz) = (t0 + line, fixed, k)
      const float sxa = skg[t0 + 2 * warp], sxb = skg[t0 + 2 * warp + 1], sy = skg[fixed];
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const float sz = skl[a * 32 + lane];
        float la, lb;
        if (q1) {
          const float my = 1.f - sy * (1.f / 6.f), mz = 1.f - sz * (1.f / 6.f);
          const float mxa = 1.f - sxa * (1.f / 6.f), mxb = 1.f - sxb * (1.f / 6.f);
          const float t = sy * mz + my * sz;
          la = -(float)kQ1Scale * (sxa * my * mz + mxa * t);
          lb = -(float)kQ1Scale * (sxb * my * mz + mxb * t);
        } else {
          la = -(sxa + sy + sz);
          lb = -(sxb + sy + sz);
        }
        const bool zero_a = (t0 + 2 * warp) == 0 && fixed == 0 && a == 0 && lane == 0;
        v[a] = make_float2(zero_a ? 0.f : v[a].x / la, v[a].y / lb);
      }
      phase_fence();
      mirror_apply<R, true>(v, lane, [&](int a, float2 y, float2 c) {   // Y_n = 0
        return inverse_input(wm[a * 32 + lane], y.x, c.x, y.y, c.y);
      });
      phase_fence();
    }
  }
  if (MODE != 0) {
    fft_warp_dit<R>(v, t1, w32, tr, lane);
    __syncwarp();
    constexpr float inv_n = 1.f / (float)n;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int s = dct_at(dct_src(lane + 32 * m, n));
      Sa[s] = v[m].x * inv_n;
      Sb[s] = -v[m].y * inv_n;
    }
  }
  __syncthreads();
  {
    float4 buf[kIt];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kDctThreads;
      if (q < kVec) {
        float e[4];
        if (axis == 0) {
          const int l = (4 * q) / n, i = (4 * q) % n;
#pragma unroll
          for (int c = 0; c < 4; ++c) e[c] = S[l * LS + dct_at(i + c)];
        } else {
          const int i = q >> 3, l = 4 * (q & 7);
#pragma unroll
          for (int c = 0; c < 4; ++c) e[c] = S[(l + c) * LS + dct_at(i)];
        }
        buf[it] = make_float4(e[0], e[1], e[2], e[3]);
      }
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kDctThreads;
      if (q < kVec) {
        const int64_t g = axis == 0 ? base + 4 * (int64_t)q : base + (q >> 3) * rstride + 4 * (q & 7);
        *reinterpret_cast<float4*>(out + g) = buf[it];
      }
    }
  }
}

// ---- n = 256: the same five passes with each complex FFT split 16 x 16
// (Stockham through shared memory) instead of a warp-wide register FFT: 16
// threads per FFT (two real lines), each holding 16 points, a DFT-16 in
// registers, a twiddle, a transpose through the FFT's own two tile rows, and
// a second DFT-16.  For p = t + 16 m and k = u + 16 k1,
//   Z_k = sum_t W16^{t k1} W256^{t u} (sum_m z_p W16^{m u}),
// so thread t forms the inner DFT over m, multiplies by W256^{t k2} and
// stores it; thread u gathers the sixteen values for its k2 = u and forms the
// outer DFT over t.  The transpose is XOR-swizzled (slot k2 * 16 + (t ^ k2)),
// so neither its stores nor its loads conflict in the banks.  An FFT's
// threads share a warp and only its own rows, so the phases need warp
// barriers only; the block synchronises around the tile's global copies.
// The DCT mapping around the FFT (Makhoul's permutation, two lines per
// complex FFT, the post-twiddle of the forward transform and the pre-twiddle
// of the inverse) is that of the warp-FFT passes.
constexpr int kD2N = 256;
constexpr int kD2Threads = 256;   // 16 FFTs (32 lines) x 16 threads

__device__ __forceinline__ void dft4_f(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = make_float2(d02.x + d13.y, d02.y - d13.x);   // d02 - i d13
  a3 = make_float2(d02.x - d13.y, d02.y + d13.x);   // d02 + i d13
}

// X_k = sum_n x_n e^{-2 pi i n k / 16}, natural order in and out: n = 4 n1 + n2,
// k = k1 + 4 k2; DFT-4 over n1, twiddle W16^{n2 k1}, DFT-4 over n2.
__device__ __forceinline__ void dft16_f(float2 (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4_f(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // x[4 k1 + n2] = A[n2][k1]; A[n2][k1] *= W16^{n2 k1}
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
  const float2 w1 = make_float2(c1, -s1), w2 = make_float2(r2, -r2), w3 = make_float2(s1, -c1);
  const float2 w6 = make_float2(-r2, -r2), w9 = make_float2(-c1, s1);
  x[4 * 1 + 1] = cmul(x[4 * 1 + 1], w1);
  x[4 * 1 + 2] = cmul(x[4 * 1 + 2], w2);
  x[4 * 1 + 3] = cmul(x[4 * 1 + 3], w3);
  x[4 * 2 + 1] = cmul(x[4 * 2 + 1], w2);
  x[4 * 2 + 2] = make_float2(x[4 * 2 + 2].y, -x[4 * 2 + 2].x);   // W16^4 = -i
  x[4 * 2 + 3] = cmul(x[4 * 2 + 3], w6);
  x[4 * 3 + 1] = cmul(x[4 * 3 + 1], w3);
  x[4 * 3 + 2] = cmul(x[4 * 3 + 2], w6);
  x[4 * 3 + 3] = cmul(x[4 * 3 + 3], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4_f(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  // x[4 k1 + k2] = X[k1 + 4 k2]: back to natural order
  float2 y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// The 256-point FFT of the 16 points z[m] = z_{t + 16 m} of this thread's FFT:
// on return z[k1] = Z_{t + 16 k1}.  sc: the FFT's scratch (256 float2).
__device__ __forceinline__ void fft256_16x16(float2 (&z)[16], float2* sc, const float2* tw, int t) {
  dft16_f(z);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) z[k2] = cmul(z[k2], tw[t * k2]);
  __syncwarp();   // the FFT's rows are read before they hold the transpose
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) sc[k2 * 16 + (t ^ k2)] = z[k2];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 16; ++m) z[m] = sc[t * 16 + (m ^ t)];
  dft16_f(z);
}

// MODE 0: forward DCT-II along `axis`; 1: its inverse; 2 (axis z): forward,
// division by the eigenvalue, inverse.  Lines as in dct_pass_kernel; a block
// takes 32 lines, `in` may be `out`.
template <int MODE>
__global__ void __launch_bounds__(kD2Threads, 3)
    dct256_pass_kernel(const float* in, float* out, int axis, const float2* __restrict__ twg,
                       const float2* __restrict__ wqg, const float* __restrict__ skg, int q1,
                       const int* __restrict__ gate) {
  constexpr int n = kD2N;
  if (*gate) return;
  __shared__ float2 tw[n];            // e^{-2 pi i j / n}
  __shared__ float2 wq[n + 1];        // e^{-i pi k / (2 n)}
  __shared__ float sk[n];             // 4 sin^2(pi k / (2 n))
  __shared__ __align__(16) float S[kDctTile * 260];
  const int tid = threadIdx.x;
  for (int q = tid; q <= n; q += kD2Threads) {
    if (q < n) {
      tw[q] = twg[q];
      if (MODE == 2) sk[q] = skg[q];
    }
    wq[q] = wqg[q];
  }
  // rows of 260 floats along x (float4-aligned copies), 257 across (the
  // transposed copies then fall in distinct banks)
  const int LS = axis == 0 ? 260 : 257;
  const int groups = n / kDctTile;
  const int fixed = blockIdx.x / groups, t0 = (blockIdx.x - fixed * groups) * kDctTile;
  const int64_t nn = (int64_t)n * n;
  const int64_t base = axis == 0 ? ((int64_t)fixed * n + t0) * n : axis == 1 ? fixed * nn + t0 : (int64_t)fixed * n + t0;
  const int64_t rstride = axis == 1 ? n : nn;
  constexpr int kVec = kDctTile * n / 4;
  constexpr int kIt = kVec / kD2Threads;   // 8 float4 per thread
  {
    float4 buf[kIt];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kD2Threads;
      const int64_t g = axis == 0 ? base + 4 * (int64_t)q : base + (q >> 3) * rstride + 4 * (q & 7);
      buf[it] = *reinterpret_cast<const float4*>(in + g);
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kD2Threads;
      if (axis == 0) {
        *reinterpret_cast<float4*>(&S[(q >> 6) * 260 + 4 * (q & 63)]) = buf[it];
      } else {
        const int i = q >> 3, l = 4 * (q & 7);
        S[(l + 0) * 257 + i] = buf[it].x;
        S[(l + 1) * 257 + i] = buf[it].y;
        S[(l + 2) * 257 + i] = buf[it].z;
        S[(l + 3) * 257 + i] = buf[it].w;
      }
    }
  }
  __syncthreads();

  const int f = tid >> 4, t = tid & 15;   // FFT f: lines 2f, 2f + 1
  float* ra = S + (2 * f) * LS;
  float* rb = ra + LS;
  float2* sc = reinterpret_cast<float2*>(ra);   // 256 float2 over the two rows
  float2 z[16];
  if (MODE != 1) {
    // forward: z_p = v_a[p] + i v_b[p], v_p = x_{2p} (p < n/2), x_{2(n-1-p)+1}
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int p = t + 16 * m;
      const int sp = p < n / 2 ? 2 * p : 2 * n - 1 - 2 * p;
      z[m] = make_float2(ra[sp], rb[sp]);
    }
    fft256_16x16(z, sc, tw, t);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sc[t + 16 * k1] = z[k1];
    __syncwarp();
    // X_k = Re(e^{-i pi k / 2n} V_k) of both lines, in pairs (k, n - k):
    // V_a = (Z_k + conj Z_{n-k}) / 2, V_b = (Z_k - conj Z_{n-k}) / 2i, and at
    // n - k the conjugates
    float xa[16], xb[16], xa128 = 0.f, xb128 = 0.f;
#pragma unroll
    for (int sidx = 0; sidx < 8; ++sidx) {
      const int k = t + 16 * sidx;
      const float2 zk = sc[k], zc = sc[(n - k) & (n - 1)];
      const float2 va = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
      const float2 vb = make_float2(0.5f * (zk.y + zc.y), 0.5f * (zc.x - zk.x));
      const float2 w = wq[k], wc = wq[n - k];
      xa[sidx] = w.x * va.x - w.y * va.y;
      xb[sidx] = w.x * vb.x - w.y * vb.y;
      xa[8 + sidx] = wc.x * va.x + wc.y * va.y;
      xb[8 + sidx] = wc.x * vb.x + wc.y * vb.y;
    }
    if (t == 0) {
      const float2 zh = sc[n / 2];
      xa128 = wq[n / 2].x * zh.x;
      xb128 = wq[n / 2].x * zh.y;
    }
    if (MODE == 2) {
      // divide by the eigenvalue of mode (kx, ky, kz) = (t0 + line, fixed, k)
      const float sxa = sk[t0 + 2 * f], sxb = sk[t0 + 2 * f + 1], sy = sk[fixed];
      auto lam = [&](float sx, float sz) {
        if (q1) {
          const float my = 1.f - sy * (1.f / 6.f), mz = 1.f - sz * (1.f / 6.f), mx = 1.f - sx * (1.f / 6.f);
          return -(float)kQ1Scale * (sx * my * mz + mx * (sy * mz + my * sz));
        }
        return -(sx + sy + sz);
      };
      // (times the correctly rounded reciprocal: the correction needs FP32
      // accuracy, not the division's last bit)
#pragma unroll
      for (int sidx = 0; sidx < 8; ++sidx) {
        const int k = t + 16 * sidx;
        const bool zero_a = (t0 + 2 * f) == 0 && fixed == 0 && k == 0;
        xa[sidx] = zero_a ? 0.f : xa[sidx] * __frcp_rn(lam(sxa, sk[k]));
        xb[sidx] = xb[sidx] * __frcp_rn(lam(sxb, sk[k]));
        const float skc = sk[(n - k) & (n - 1)];   // at k = 0 the value is not used (n - k = n)
        xa[8 + sidx] = xa[8 + sidx] * __frcp_rn(lam(sxa, skc));
        xb[8 + sidx] = xb[8 + sidx] * __frcp_rn(lam(sxb, skc));
      }
      if (t == 0) {
        xa128 = xa128 * __frcp_rn(lam(sxa, sk[n / 2]));
        xb128 = xb128 * __frcp_rn(lam(sxb, sk[n / 2]));
      }
    }
    __syncwarp();   // every thread has read its Z before the rows take X
#pragma unroll
    for (int sidx = 0; sidx < 8; ++sidx) {
      const int k = t + 16 * sidx;
      ra[k] = xa[sidx];
      rb[k] = xb[sidx];
      if (k) {
        ra[n - k] = xa[8 + sidx];
        rb[n - k] = xb[8 + sidx];
      }
    }
    if (t == 0) {
      ra[n / 2] = xa128;
      rb[n / 2] = xb128;
    }
  }
  if (MODE != 0) {
    __syncwarp();
    // inverse: the FFT of conj(V_a + i V_b), conj V_k = e^{-i pi k / 2n} (X_k + i X_{n-k})
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int p = t + 16 * m;
      const float xa = ra[p], xb = rb[p];
      const float xan = p ? ra[n - p] : 0.f, xbn = p ? rb[n - p] : 0.f;
      z[m] = inverse_input(wq[p], xa, xan, xb, xbn);
    }
    fft256_16x16(z, sc, tw, t);
    __syncwarp();
    // v_a + i v_b = conj(Z) / n, back in place: x_{2q} = v_q, x_{2(n-1-q)+1} = v_q
    constexpr float inv_n = 1.f / (float)n;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
      const int q = t + 16 * k1;
      const int sq = q < n / 2 ? 2 * q : 2 * n - 1 - 2 * q;
      ra[sq] = z[k1].x * inv_n;
      rb[sq] = -z[k1].y * inv_n;
    }
  }
  __syncthreads();
  {
    float4 buf[kIt];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kD2Threads;
      if (axis == 0) {
        buf[it] = *reinterpret_cast<const float4*>(&S[(q >> 6) * 260 + 4 * (q & 63)]);
      } else {
        const int i = q >> 3, l = 4 * (q & 7);
        buf[it] = make_float4(S[(l + 0) * 257 + i], S[(l + 1) * 257 + i], S[(l + 2) * 257 + i],
                              S[(l + 3) * 257 + i]);
      }
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int q = tid + it * kD2Threads;
      const int64_t g = axis == 0 ? base + 4 * (int64_t)q : base + (q >> 3) * rstride + 4 * (q & 7);
      *reinterpret_cast<float4*>(out + g) = buf[it];
    }
  }
}

template <int R>
int spectral_passes(wgeo_handle* h, float* e, const float* r, const int* gate, cudaStream_t s) {
  constexpr int n = 32 * R;
  if (n == kD2N) {
    const int blocks = n * (n / kDctTile);
    const int q1 = h->opt.galerkin ? 1 : 0;
#define WGEO_DCT256_PASS(MODE, SRC, AXIS)                                                                 \
  dct256_pass_kernel<MODE><<<blocks, kD2Threads, 0, s>>>(SRC, e, AXIS, h->dct_tw, h->dct_wq, h->dct_sk, q1, \
                                                         gate);                                          \
  WGEO_LAUNCH_CHECK();
    WGEO_DCT256_PASS(0, r, 0)
    WGEO_DCT256_PASS(0, e, 1)
    WGEO_DCT256_PASS(2, e, 2)
    WGEO_DCT256_PASS(1, e, 1)
    WGEO_DCT256_PASS(1, e, 0)
#undef WGEO_DCT256_PASS
    return WGEO_OK;
  }
  constexpr size_t smem = dct_smem<R>();
  const int blocks = n * (n / kDctTile);
  const int q1 = h->opt.galerkin ? 1 : 0;
#define WGEO_DCT_PASS(MODE, SRC, AXIS)                                                                  \
  dct_pass_kernel<R, MODE><<<blocks, kDctThreads, smem, s>>>(SRC, e, AXIS, h->dct_t1, h->dct_w32,     \
                                                              h->dct_wml, h->dct_tr, h->dct_sk,      \
                                                              h->dct_skl, q1, gate);                 \
  WGEO_LAUNCH_CHECK();
  WGEO_DCT_PASS(0, r, 0)
  WGEO_DCT_PASS(0, e, 1)
  WGEO_DCT_PASS(2, e, 2)
  WGEO_DCT_PASS(1, e, 1)
  WGEO_DCT_PASS(1, e, 0)
#undef WGEO_DCT_PASS
  return WGEO_OK;
}

// e = the solution of L e = r - mean(r) (L the handle's operator), zero mean.
int spectral_solve(wgeo_handle* h, int n, float* e, const float* r, const int* gate, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(e) | reinterpret_cast<uintptr_t>(r)) & 15) return WGEO_ERR_INVALID_ARG;
  switch (n) {
    case 32: return spectral_passes<1>(h, e, r, gate, s);
    case 64: return spectral_passes<2>(h, e, r, gate, s);
    case 128: return spectral_passes<4>(h, e, r, gate, s);
    case 256: return spectral_passes<8>(h, e, r, gate, s);
    case 512: return spectral_passes<16>(h, e, r, gate, s);
    default: return WGEO_ERR_INVALID_ARG;
  }
}

template <int R>
cudaError_t dct_attr() {
  const int mx = (int)dct_smem<R>();
  cudaError_t err = cudaFuncSetAttribute(dct_pass_kernel<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(dct_pass_kernel<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(dct_pass_kernel<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return err;
}

// The twiddle and eigenvalue tables for n, and the shared-memory opt-in of the
// pass kernels on the handle's device (host calls, kept out of any capture).
int spectral_setup(wgeo_handle* h, int n, cudaStream_t s) {
  if (!h->dct_attr) {
    WGEO_CUDA_TRY(dct_attr<1>());
    WGEO_CUDA_TRY(dct_attr<2>());
    WGEO_CUDA_TRY(dct_attr<4>());
    WGEO_CUDA_TRY(dct_attr<8>());
    WGEO_CUDA_TRY(dct_attr<16>());
    h->dct_attr = true;
  }
  if (h->dct_n != n) {
    dct_tables_kernel<<<div_up(n > 160 ? n + 1 : 161, 256), 256, 0, s>>>(n, h->dct_t1, h->dct_w32, h->dct_wml,
                                                                         h->dct_tr, h->dct_sk, h->dct_skl,
                                                                         h->dct_tw, h->dct_wq);
    WGEO_LAUNCH_CHECK();
    h->dct_n = n;
  }
  return WGEO_OK;
}

// One V-cycle for L' on level l, in place: damped Jacobi sweeps (ping-pong
// through the level's t buffer; t0 on level 0), the same transfers, the
// 8-colour small-grid kernel at 16^3 and below.
int vcycle_q1(wgeo_handle* h, int l, float* x0, const float* b0, const float* shift0, bool zero0, float* t0,
              const int* gate, cudaStream_t s) {
  const int n = h->levels[l].n;
  float* x = (l == 0) ? x0 : h->levels[l].x;
  float* t = (l == 0) ? t0 : h->levels[l].t;
  const float* b = (l == 0) ? b0 : h->levels[l].b;
  const float* shift = (l == 0) ? shift0 : nullptr;
  if (n <= kSmallN || l == h->nlevels - 1) {
    small_vcycle_q1_kernel<<<1, 1024, 0, s>>>(x, b, shift, n, gate);
    WGEO_LAUNCH_CHECK();
    return WGEO_OK;
  }
  const bool zero = (l == 0) ? zero0 : true;
  const int nc = n >> 1;
  const dim3 blk(kSX, kSY);
  const dim3 gcell(div_up(n, kSX), div_up(n, kSY), n);
  const dim3 gf(div_up(nc, kSX), div_up(n, kSY), n);      // fine pairs (prolongation)
  const dim3 gc(div_up(nc, kSX), div_up(nc, kSY), nc);
  // kNu sweeps x -> t -> x (kNu even)
  static_assert(kNu % 2 == 0, "Jacobi ping-pong ends in x");
  for (int sw = 0; sw < kNu; ++sw) {
    const float* src = (sw & 1) ? t : x;
    float* dst = (sw & 1) ? x : t;
    if (zero && sw == 0)
      jacobi_q1_kernel<true><<<gcell, blk, 0, s>>>(src, dst, b, shift, n, gate);
    else
      jacobi_q1_kernel<false><<<gcell, blk, 0, s>>>(src, dst, b, shift, n, gate);
    WGEO_LAUNCH_CHECK();
  }
  restrict_q1_kernel<<<gc, blk, 0, s>>>(x, b, shift, n, h->levels[l + 1].b, gate);
  WGEO_LAUNCH_CHECK();
  int rc = vcycle_q1(h, l + 1, x0, b0, shift0, zero0, t0, gate, s);
  if (rc) return rc;
  prolong_pair_kernel<<<gf, blk, 0, s>>>(h->levels[l + 1].x, x, n, gate);
  WGEO_LAUNCH_CHECK();
  for (int sw = 0; sw < kNu; ++sw) {
    const float* src = (sw & 1) ? t : x;
    float* dst = (sw & 1) ? x : t;
    jacobi_q1_kernel<false><<<gcell, blk, 0, s>>>(src, dst, b, shift, n, gate);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

// One solve (mode 0: forward, 1: adjoint) is a head -- the first residual
// and convergence test -- followed by loop iterations, each a correction and
// a new residual and test.  part 0 enqueues the head, part 1 one iteration.
// step: the host's step number (fixed sequence) or -1 (recorded loop body,
// counted on the device); hc / cond: the recorded loop's condition.
int enqueue_part(wgeo_handle* h, int res, int mode, int part, int step, cudaGraphConditionalHandle hc, int cond,
                 cudaStream_t s) {
  const int64_t N = (int64_t)res * res * res;
  SolveState* ss = mode == 0 ? &h->dstate->fwd : &h->dstate->bwd;
  const int* gate = &ss->done;
  const bool fp32 = (mode == 0 && h->opt.precision == WGEO_PREC_FP32);
  const int rb = grid_blocks(N, kThreads, kPartials);
  if (fp32) {
    if (part == 1) {
      // plain FP32: on spectral grids one direct FP32 solve of L x = b - mean(b)
      // (no refinement), else one FP32 V-cycle on x in place
      int rc = use_spectral(h, res) ? spectral_solve(h, res, h->chi32, h->b32, gate, s)
                                    : vcycle(h, 0, h->chi32, h->b32, &ss->bmean32, false, gate, s);
      if (rc) return rc;
    }
    residual32_kernel<<<rb, kThreads, 0, s>>>(h->chi32, h->b32, &ss->bmean32, res, h->partials, gate);
    WGEO_LAUNCH_CHECK();
    finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss, h->dstate, h->opt.tol_rel, step, 1, 0, hc, cond);
    WGEO_LAUNCH_CHECK();
    return WGEO_OK;
  }
  const double tol = mode == 0 ? h->opt.tol_rel : h->opt.tol_rel_adjoint;
  PairFF xp;
  xp.buf[0] = mode == 0 ? h->chiff[0] : h->lamff[0];
  xp.buf[1] = mode == 0 ? h->chiff[1] : h->lamff[1];
  float* x32 = mode == 0 ? h->chi32 : h->lam32;
  if (part == 1) {
    // correction: V-cycles on L e = r - mean(r)
    if (use_spectral(h, res)) {
      int rc = spectral_solve(h, res, h->e32, h->r32, gate, s);
      if (rc) return rc;
    } else {
      for (int v = 0; v < h->opt.vcycles_per_refine; ++v) {
        int rc = h->opt.galerkin ? vcycle_q1(h, 0, h->e32, h->r32, &ss->rmean32, v == 0, x32, gate, s)
                                 : vcycle(h, 0, h->e32, h->r32, &ss->rmean32, v == 0, gate, s);
        if (rc) return rc;
      }
    }
  }
  const float* e = part == 0 ? nullptr : h->e32;
  // the lumped float-float pass marches kResZ planes per block in z; the
  // unlumped and FP64 passes take one plane per block
  const bool marching = !h->opt.galerkin && !(mode == 0 && h->opt.precision == WGEO_PREC_FP64);
  const dim3 rg(div_up(div_up(res, 2), kSX), div_up(res, kSY), marching ? div_up(res, kResZ) : res);
  const int nrb = (int)(rg.x * rg.y * rg.z);
  if (h->opt.galerkin) {
    if (mode == 0)
      update_residual_q1_kernel<float><<<rg, dim3(kSX, kSY), 0, s>>>(xp, e, h->b32, res, h->r32, x32, h->partials,
                                                                     ss);
    else
      update_residual_q1_kernel<double><<<rg, dim3(kSX, kSY), 0, s>>>(xp, e, h->dchi64, res, h->r32, x32,
                                                                      h->partials, ss);
  } else if (mode == 0 && h->opt.precision == WGEO_PREC_FP64) {
    PairD xd;
    xd.buf[0] = reinterpret_cast<double*>(xp.buf[0]);
    xd.buf[1] = reinterpret_cast<double*>(xp.buf[1]);
    update_residual_f64_kernel<<<rg, dim3(kSX, kSY), 0, s>>>(xd, e, h->b32, res, h->r32, x32, h->partials, ss);
  } else if (mode == 0) {
    update_residual_kernel<float><<<rg, dim3(kSX, kSY), 0, s>>>(xp, e, h->b32, res, h->r32, x32, h->partials, ss);
  } else {
    update_residual_kernel<double><<<rg, dim3(kSX, kSY), 0, s>>>(xp, e, h->dchi64, res, h->r32, x32, h->partials,
                                                                 ss);
  }
  WGEO_LAUNCH_CHECK();
  finalize_kernel<<<1, 1024, 0, s>>>(h->partials, nrb, N, ss, h->dstate, tol, step, 0, e ? 1 : 0, hc, cond);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

int max_steps(const wgeo_handle* h, int mode) {
  return (mode == 0 && h->opt.precision == WGEO_PREC_FP32) ? h->opt.max_vcycles : h->opt.max_refine;
}

// The fixed launch sequence: the head and max_steps gated iterations.
int enqueue_solve(wgeo_handle* h, int res, int mode, bool skip, cudaStream_t s) {
  int rc = skip ? WGEO_OK : enqueue_part(h, res, mode, 0, 0, 0, 0, s);
  for (int it = 1; it <= max_steps(h, mode) && rc == WGEO_OK; ++it)
    rc = enqueue_part(h, res, mode, 1, it, 0, 0, s);
  return rc;
}

// Records the solve as a graph: the head, then a conditional WHILE node whose
// body (one iteration) runs until the convergence test clears the condition,
// so no launch happens after convergence.  Counts: the head's launches are
// returned in *head, one body's in *body.
// skip: no head (see skip_head); the loop's condition then starts at 1.
int record_solve(wgeo_handle* h, int res, int mode, bool skip, cudaGraph_t* out, long long* head,
                 long long* body) {
  cudaStream_t cs = h->capture_stream;
  cudaGraph_t g = nullptr;
  WGEO_CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hc;
  cudaError_t e = skip ? cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault)
                       : cudaGraphConditionalHandleCreate(&hc, g, 0, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return WGEO_ERR_CUDA;
  }
  long long t0 = t_kernel_launches;
  int rc = WGEO_OK;
  std::vector<cudaGraphNode_t> deps;
  if (!skip) {
    e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    rc = e == cudaSuccess ? enqueue_part(h, res, mode, 0, 0, hc, 1, cs) : WGEO_ERR_CUDA;
  }
  if (!skip && e == cudaSuccess) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &d, nullptr, &nd) == cudaSuccess)
      deps.assign(d, d + nd);
    cudaGraph_t gg = g;
    if (cudaStreamEndCapture(cs, &gg) != cudaSuccess && rc == WGEO_OK) rc = WGEO_ERR_CUDA;
  }
  *head = t_kernel_launches - t0;
  cudaGraph_t bodyg = nullptr;
  if (rc == WGEO_OK) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps.data(), nullptr, deps.size(), &p) != cudaSuccess)
      rc = WGEO_ERR_CUDA;
    else
      bodyg = p.conditional.phGraph_out[0];
  }
  t0 = t_kernel_launches;
  if (rc == WGEO_OK) {
    e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      rc = WGEO_ERR_CUDA;
    } else {
      rc = enqueue_part(h, res, mode, 1, -1, hc, 1, cs);
      cudaGraph_t bb = bodyg;
      if (cudaStreamEndCapture(cs, &bb) != cudaSuccess && rc == WGEO_OK) rc = WGEO_ERR_CUDA;
    }
  }
  *body = t_kernel_launches - t0;
  if (rc != WGEO_OK) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return rc;
  }
  *out = g;
  return WGEO_OK;
}

}  // namespace

long long loop_launches() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_loop_launches, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (long long)v;
}

int coarsest_size(int res) {
  int n = res;
  while ((n % 2) == 0 && n > 8) n /= 2;
  return n;
}

int build_levels(wgeo_handle* h, int res) {
  int n = res;
  int l = 0;
  float* pool = h->level_pool;
  h->levels[0].n = n;
  h->levels[0].x = nullptr;
  h->levels[0].b = nullptr;
  h->levels[0].t = nullptr;
  while ((n % 2) == 0 && n > 8) {
    n /= 2;
    ++l;
    if (l >= kMaxLevels) return WGEO_ERR_INVALID_ARG;
    const int64_t M = (int64_t)n * n * n;
    const int64_t Ma = (M + 63) / 64 * 64;
    h->levels[l].n = n;
    h->levels[l].x = pool;
    h->levels[l].b = pool + Ma;
    h->levels[l].t = h->opt.galerkin ? pool + 2 * Ma : nullptr;
    pool += (h->opt.galerkin ? 3 : 2) * Ma;
  }
  if (n > 16) return WGEO_ERR_INVALID_ARG;
  h->nlevels = l + 1;
  return WGEO_OK;
}

int launch_solve_body(wgeo_handle* h, int res, int mode, bool cold, cudaStream_t s);

// A solve from zero with the lumped operator, the spectral correction and the
// float-float iterate needs no head: its first residual is b itself, so the
// first correction reads b (copied, or rounded from the adjoint's FP64 b, into
// the residual buffer) and the first iteration's pass takes x as 0 (the cold
// flag stays set until its test).  The iterations and their results are those
// of the solve with the head.
bool skip_head(const wgeo_handle* h, int res, int mode, bool cold) {
  return cold && use_spectral(h, res) && !h->opt.galerkin && (mode == 1 || h->opt.precision == WGEO_PREC_MIXED);
}

// Enqueues one solve.  The launch sequence depends only on (res, mode,
// options), and every pointer it uses is owned by the handle, so it is
// recorded once as a CUDA graph and replayed; while the caller's stream is
// itself being captured the kernels are enqueued directly instead.
int launch_solve(wgeo_handle* h, int res, int mode, bool cold, cudaStream_t s) {
  const int64_t N = (int64_t)res * res * res;
  SolveState* ss = mode == 0 ? &h->dstate->fwd : &h->dstate->bwd;
  if (use_spectral(h, res)) {
    int rc = spectral_setup(h, res, s);
    if (rc) return rc;
  }
  const bool skip = skip_head(h, res, mode, cold);
  if (mode == 1) {
    const int rb = grid_blocks(N, kThreads, kPartials);
    if (h->opt.galerkin) {
      // the adjoint system L lambda = dchi, written for L' = 12 L
      scale64_kernel<<<grid_blocks(N, kThreads, 152 * 16), kThreads, 0, s>>>(h->dchi64, N, (double)kQ1Scale);
      WGEO_LAUNCH_CHECK();
    }
    rhs_stats64_kernel<<<rb, kThreads, 0, s>>>(h->dchi64, N, h->partials, skip ? h->r32 : nullptr);
    WGEO_LAUNCH_CHECK();
    rhs_stats_finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss);
    WGEO_LAUNCH_CHECK();
  }
  // native FP64 iterate: a warm start's float-float pair becomes a double
  // first, and the solution becomes a pair again after the solve
  const bool f64 = (mode == 0 && h->opt.precision == WGEO_PREC_FP64);
  PairD xd;
  xd.buf[0] = reinterpret_cast<double*>(h->chiff[0]);
  xd.buf[1] = reinterpret_cast<double*>(h->chiff[1]);
  if (f64 && !cold) {
    f64_from_ff_kernel<<<grid_blocks(N, 256, 152 * 16), 256, 0, s>>>(xd, ss, N);
    WGEO_LAUNCH_CHECK();
  }
  int rc = launch_solve_body(h, res, mode, cold, s);
  if (rc) return rc;
  if (f64) {
    ff_from_f64_kernel<<<grid_blocks(N, 256, 152 * 16), 256, 0, s>>>(xd, ss, N);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

// The solve proper (see launch_solve): the recorded graph or the fixed sequence.
int launch_solve_body(wgeo_handle* h, int res, int mode, bool cold, cudaStream_t s) {
  SolveState* ss = mode == 0 ? &h->dstate->fwd : &h->dstate->bwd;
  const bool fp32_plain = (mode == 0 && h->opt.precision == WGEO_PREC_FP32);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  WGEO_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  const int steps = max_steps(h, mode);
  // the direct correction reaches the float-float limit in two steps (the
  // first is exact to FP32 rounding): always take both, so that chi, and the
  // adjoint's right-hand side built from it, carry no solver error
  // (plain FP32 takes its one direct solve)
  const int min_steps = use_spectral(h, res) ? (fp32_plain ? 1 : 2) : 0;
  const bool skip = skip_head(h, res, mode, cold);
  if (skip && mode == 0)
    WGEO_CUDA_TRY(cudaMemcpyAsync(h->r32, h->b32, sizeof(float) * (size_t)res * res * res, cudaMemcpyDeviceToDevice, s));
  if (!h->opt.use_graphs || cap != cudaStreamCaptureStatusNone) {
    solve_begin_kernel<<<1, 1, 0, s>>>(ss, cold ? 1 : 0, steps, min_steps, 0);
    WGEO_LAUNCH_CHECK();
    return enqueue_solve(h, res, mode, skip, s);
  }
  SolverGraph& g = h->graphs[2 * mode + (skip ? 1 : 0)];
  const int gmode = mode * 3 + (mode == 0 ? h->opt.precision : 0);
  if (g.exec == nullptr || g.res != res || g.mode != gmode) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (!h->capture_stream) WGEO_CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    long long head = 0, body = 0;
    int rc = record_solve(h, res, mode, skip, &graph, &head, &body);
    // recorded, not run: the head is counted at each replay, the body on the
    // device once per iteration
    t_kernel_launches -= head + body;
    g_kernel_launches.fetch_sub(head + body, std::memory_order_relaxed);
    if (rc) return rc;
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return WGEO_ERR_CUDA;
    }
    g.res = res;
    g.mode = gmode;
    g.launches = head;
    g.body_launches = body;
  }
  solve_begin_kernel<<<1, 1, 0, s>>>(ss, cold ? 1 : 0, steps, min_steps, (int)g.body_launches);
  WGEO_LAUNCH_CHECK();
  WGEO_CUDA_TRY(cudaGraphLaunch(g.exec, s));
  g_kernel_launches.fetch_add(g.launches, std::memory_order_relaxed);
  t_kernel_launches += g.launches;
  return WGEO_OK;
}

}  // namespace wgeo
