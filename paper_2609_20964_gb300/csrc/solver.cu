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
// Plain FP32 (comparator): V-cycles directly on x32 with an FP32 residual.
//
// Multigrid: cell-centred, halving while even and larger than 8; red-black
// Gauss-Seidel, 2 pre- and 2 post-sweeps; residual restricted with weight 1/2
// on the 8 children (average x H^2/h^2 for the unit-free operator); trilinear
// prolongation (3/4, 1/4 per axis, mirrored at the walls).  Levels with
// n >= 128 use two fused z-marching kernels per V-cycle: a CTA owns a 64 x 16
// column tile and a 16-plane z chunk, keeps a ring of planes in shared memory
// (next plane prefetched with cp.async) and pipelines the four half-sweeps
// (half-sweep s works s planes behind the newest), which reproduces global
// red-black Gauss-Seidel exactly while x is read from HBM once; the
// pre-smoothing kernel also forms the residual and restricts it, the
// post-smoothing kernel adds the prolonged coarse correction while loading.
// Mid-size levels use one launch per half-sweep; grids of at most 16^3 run a
// whole V-cycle hierarchy in one CTA's shared memory.
//
// Every kernel of the fixed launch sequence reads the solve's `done` flag and
// returns at once when it is set, so the sequence (recorded once as a CUDA
// graph) stops doing work as soon as the tolerance is met.
#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

constexpr int kThreads = 256;
constexpr int kNu = 2;              // red-black sweeps before and after the coarse correction
constexpr int kTX = 64, kTY = 16;
constexpr int kSmThreads = 512;
constexpr int kSmallN = 16;         // levels up to 16^3 are solved in one CTA

__device__ __forceinline__ int64_t lin(int i, int j, int k, int n) {
  return ((int64_t)k * n + j) * n + i;
}

struct PairFF {
  float2* buf[2];
};

__device__ __forceinline__ float rhs_hi(const float* b, int64_t t, float& lo) {
  lo = 0.f;
  return b[t];
}
__device__ __forceinline__ float rhs_hi(const double* b, int64_t t, float& lo) {
  const double v = b[t];
  const float hi = (float)v;
  lo = (float)(v - (double)hi);
  return hi;
}

// ---------------------------------------------------------------- refinement pass
// The refinement iterate is kept in float-float (hi + lo, ~48-bit significand):
// on this GPU the FP64 pipe made an FP64 stencil pass about 12x slower than its
// memory traffic, while the error-free sums below run on the FP32 pipe.
//   x_new = x + e (e may be null: no correction this step; cold: x := 0),
//   x32 = hi(x_new), r32 = b - L x_new (each neighbour difference formed
//   exactly), per-thread sums of r and r^2 in FP32, per-block sums in FP64.
template <typename TB>
__global__ void update_residual_kernel(PairFF xp, const float* __restrict__ e, const TB* __restrict__ b,
                                       int n, float* __restrict__ r32, float* __restrict__ x32,
                                       double* __restrict__ partials, SolveState* ss) {
  if (ss->done) return;
  __shared__ double red[32];
  const int cur = ss->xidx;
  const bool cold = ss->cold != 0;
  const float2* __restrict__ xin = xp.buf[cur];
  float2* __restrict__ xout = xp.buf[e ? cur ^ 1 : cur];
  const int64_t N = (int64_t)n * n * n;
  float s1 = 0.f, s2 = 0.f;
  (void)N;
  for (int row = blockIdx.x; row < n * n; row += gridDim.x) {     // rows (j, k), x along threads
   const int j = row % n, k = row / n;
   for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t t = (int64_t)row * n + i;
    float2 xc = make_float2(0.f, 0.f), acc = make_float2(0.f, 0.f);
    if (!cold) {
      auto val = [&](int64_t q) {
        const float2 v = xin[q];
        return e ? ff_add_f(v, e[q]) : v;
      };
      xc = val(t);
      if (i > 0) acc = ff_add(acc, ff_sub(val(t - 1), xc));
      if (i < n - 1) acc = ff_add(acc, ff_sub(val(t + 1), xc));
      if (j > 0) acc = ff_add(acc, ff_sub(val(t - n), xc));
      if (j < n - 1) acc = ff_add(acc, ff_sub(val(t + n), xc));
      if (k > 0) acc = ff_add(acc, ff_sub(val(t - (int64_t)n * n), xc));
      if (k < n - 1) acc = ff_add(acc, ff_sub(val(t + (int64_t)n * n), xc));
    }
    float blo;
    const float bhi = rhs_hi(b, t, blo);
    const float2 r = ff_sub(make_float2(bhi, blo), acc);
    if (e || cold) xout[t] = xc;
    x32[t] = xc.x;
    const float rf = r.x + r.y;
    r32[t] = rf;
    s1 += rf;
    s2 += rf * rf;
   }
  }
  double d1 = block_sum<kThreads>((double)s1, red);
  double d2 = block_sum<kThreads>((double)s2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = d1;
    partials[2 * blockIdx.x + 1] = d2;
  }
}

__global__ void residual32_kernel(const float* __restrict__ x, const float* __restrict__ b,
                                  const double* __restrict__ shift, int n,
                                  double* __restrict__ partials, const int* __restrict__ gate) {
  if (*gate) return;
  __shared__ float red[32];
  const int64_t N = (int64_t)n * n * n;
  const float sh = (float)*shift;
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
__global__ void finalize_kernel(const double* __restrict__ partials, int nblocks, int64_t N,
                                SolveState* ss, DevState* st, double tol, int step, int last, int fp32,
                                int flip) {
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
    if (flip) ss->xidx ^= 1;
    ss->cold = 0;
    const double mean = s1 / (double)N;
    const double rn = sqrt(fmax(s2 - s1 * mean, 0.0));
    ss->rmean = mean;
    const double bn = ss->bnorm;
    const double rel = (bn > 0.0) ? rn / bn : 0.0;
    ss->rel = rel;
    ss->iter = step;
    if (bn <= 0.0 || rel <= tol) {
      ss->done = 1;
    } else if (last) {
      atomicOr(&st->status, WGEO_STATUS_NOT_CONVERGED);
      ss->done = 1;
    }
  }
}

__global__ void solve_begin_kernel(SolveState* ss, int cold) {
  ss->done = 0;
  ss->iter = 0;
  ss->rel = 0.0;
  ss->rmean = 0.0;
  ss->cold = cold;
}

// ---------------------------------------------------------------- fused smoothers
// Levels with n >= kFusedMin.  A CTA owns a kTX x kTY column tile and a
// kZC-plane z chunk and walks z, keeping a ring of x planes (with halo) in
// shared memory; the next plane is prefetched with cp.async while the current
// one is processed.  Half-sweep s of the pipeline works s planes behind the
// newest plane, so every update sees exactly the neighbour values a global
// red-black Gauss-Seidel sweep would.  b is read through the L1/L2 caches.
constexpr int kFusedMin = 128;

template <bool PRE>
struct SmGeom {
  static constexpr int H = PRE ? 2 * kNu + 1 : 2 * kNu;   // halo of the loaded tile
  static constexpr int WX = kTX + 2 * H, WY = kTY + 2 * H, P = WX * WY;
  static constexpr int RX = PRE ? 2 * kNu + 4 : 2 * kNu + 3; // planes alive + 1 prefetch slot
  static constexpr int CW = WX / 2 + 3, CH = WY / 2 + 3;       // coarse staging window (POST)
  static constexpr size_t smem =
      sizeof(float) * ((size_t)RX * P + (PRE ? (kTX / 2) * (kTY / 2) : CW * CH));
};

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

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// PRE: x_out = 2 red-black sweeps (red first) of x_in (or of 0 when ZERO), and
//      bc = 1/2 * sum of the children residuals b - L x_out.
// POST: x_out = 2 sweeps (black first) of x_in + P xc.
template <bool PRE, bool ZERO>
__global__ void __launch_bounds__(kSmThreads, 2) smooth_kernel(const float* __restrict__ xin,
                                                               float* __restrict__ xout,
                                                               const float* __restrict__ b,
                                                               const double* __restrict__ shift, int n, int zc,
                                                               const float* __restrict__ xc,
                                                               float* __restrict__ bc,
                                                               const int* __restrict__ gate) {
  if (*gate) return;
  using G = SmGeom<PRE>;
  constexpr int NPAIR = G::P / 2;                               // cell pairs per plane (WX even)
  constexpr int SLOTS = (NPAIR + kSmThreads - 1) / kSmThreads;  // pairs per thread
  extern __shared__ float sm[];
  float* xs = sm;                       // RX planes
  float* cacc = sm + G::RX * G::P;      // coarse accumulator (PRE) / coarse staging (POST)
  const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, n);
  const int ax = max(X0 - G::H, 0), bx = min(X0 + kTX + G::H, n);
  const int ay = max(Y0 - G::H, 0), by = min(Y0 + kTY + G::H, n);
  const int zlo = max(z0 - G::H, 0), zhi = min(z1 + G::H, n);
  const float sh = shift ? (float)*shift : 0.f;
  const int nc = n >> 1;
  const int64_t nn = (int64_t)n * n;
  const int c0 = PRE ? 0 : 1;           // colour of the first half-sweep
  const int zend = zhi + 2 * kNu + (PRE ? 1 : 0);

  // Per-thread cell table, built once.  Within one z step every half-sweep s
  // works on plane zin - s with colour c0 ^ (s-1), so the cell of a pair that
  // has the right colour depends only on (row, zin): phase = rowph ^ (zin & 1).
  int cloc[SLOTS][2], boff[SLOTS][2], info[SLOTS][2];   // info: depth | neighbour mask << 8
  int rowph[SLOTS];
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const int pr = threadIdx.x + k * kSmThreads;
    const int ly = pr / (G::WX / 2), j = pr % (G::WX / 2);
    const int gy = Y0 - G::H + ly;
    rowph[k] = (c0 - 1 + gy + X0 + G::H) & 1;
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
      const int lx = 2 * j + ph, gx = X0 - G::H + lx;
      cloc[k][ph] = ly * G::WX + lx;
      boff[k][ph] = gy * n + gx;
      int depth = -1;
      if (pr < NPAIR && gx >= ax && gx < bx && gy >= ay && gy < by) {
        depth = 2 * kNu;
        if (ax > 0) depth = min(depth, gx - ax);
        if (bx < n) depth = min(depth, bx - 1 - gx);
        if (ay > 0) depth = min(depth, gy - ay);
        if (by < n) depth = min(depth, by - 1 - gy);
      }
      const int mask = (gx > 0 ? 1 : 0) | (gx < n - 1 ? 2 : 0) | (gy > 0 ? 4 : 0) | (gy < n - 1 ? 8 : 0);
      info[k][ph] = depth | (mask << 8);
    }
  }

  auto issue = [&](int z) {             // start loading plane z into its ring slot
    float* xp = xs + (z % G::RX) * G::P;
    const float* src = xin + (int64_t)z * nn;
    for (int c = threadIdx.x; c < G::P; c += blockDim.x) {
      const int gx = X0 - G::H + c % G::WX, gy = Y0 - G::H + c / G::WX;
      const bool in = gx >= ax && gx < bx && gy >= ay && gy < by;
      if (in && !ZERO)
        cp_async4(xp + c, src + gy * n + gx);
      else
        xp[c] = 0.f;
    }
  };

  issue(zlo);
  cp_async_commit();
  for (int zin = zlo; zin < zend; ++zin) {
    if (zin + 1 < zhi) issue(zin + 1);
    cp_async_commit();
    cp_async_wait1();                   // plane zin has landed (this thread's copies)
    if (!PRE && zin < zhi) {
      // prolongation, separably: the coarse window interpolated in z into shared
      // memory (2 reads per coarse cell), then bilinear in x, y from there
      float* cz = cacc;
      const int K = zin >> 1;
      const int K2 = min(max((zin & 1) ? K + 1 : K - 1, 0), nc - 1);
      const int cI0 = ((X0 - G::H) >> 1) - 1, cJ0 = ((Y0 - G::H) >> 1) - 1;
      const float* xk = xc + (int64_t)K * nc * nc;
      const float* xk2 = xc + (int64_t)K2 * nc * nc;
      for (int c = threadIdx.x; c < G::CW * G::CH; c += blockDim.x) {
        const int ci = min(max(cI0 + c % G::CW, 0), nc - 1);
        const int cj = min(max(cJ0 + c / G::CW, 0), nc - 1);
        cz[c] = 0.75f * xk[cj * nc + ci] + 0.25f * xk2[cj * nc + ci];
      }
      __syncthreads();
      float* xp = xs + (zin % G::RX) * G::P;
      for (int c = threadIdx.x; c < G::P; c += blockDim.x) {
        const int gx = X0 - G::H + c % G::WX, gy = Y0 - G::H + c / G::WX;
        if (gx >= ax && gx < bx && gy >= ay && gy < by) {
          const int I = gx >> 1, J = gy >> 1;
          const int I2 = min(max((gx & 1) ? I + 1 : I - 1, 0), nc - 1);
          const int J2 = min(max((gy & 1) ? J + 1 : J - 1, 0), nc - 1);
          const int r1 = (J - cJ0) * G::CW, r2 = (J2 - cJ0) * G::CW;
          xp[c] += 0.5625f * cz[r1 + I - cI0] + 0.1875f * cz[r1 + I2 - cI0] +
                   0.1875f * cz[r2 + I - cI0] + 0.0625f * cz[r2 + I2 - cI0];
        }
      }
    }
    __syncthreads();
    const int zph = zin & 1;
#pragma unroll
    for (int s = 1; s <= 2 * kNu; ++s) {
      const int p = zin - s;
      const int plo = zlo + (zlo > 0 ? s : 0), phi = zhi - (zhi < n ? s : 0);
      if (p >= plo && p < phi) {
        float* xp = xs + (p % G::RX) * G::P;
        const float* xm = xs + ((p + G::RX - 1) % G::RX) * G::P;
        const float* xq = xs + ((p + 1) % G::RX) * G::P;
        const bool hm = p > 0, hq = p < n - 1;
        const float* bp = b + (int64_t)p * nn;
        const int zcnt = (hm ? 1 : 0) + (hq ? 1 : 0);
#pragma unroll
        for (int k = 0; k < SLOTS; ++k) {
          const int ph = rowph[k] ^ zph;
          const int inf = ph ? info[k][1] : info[k][0];     // selects keep the tables in registers
          if ((inf & 0xff) < s || (inf & 0x80)) continue;   // outside this stage's region / domain
          const int c = ph ? cloc[k][1] : cloc[k][0];
          const int bo = ph ? boff[k][1] : boff[k][0];
          const int m = inf >> 8;
          float acc = 0.f;
          int cnt = zcnt;
          if (m & 1) { acc += xp[c - 1]; ++cnt; }
          if (m & 2) { acc += xp[c + 1]; ++cnt; }
          if (m & 4) { acc += xp[c - G::WX]; ++cnt; }
          if (m & 8) { acc += xp[c + G::WX]; ++cnt; }
          if (hm) acc += xm[c];
          if (hq) acc += xq[c];
          xp[c] = __fdividef(acc - (__ldg(bp + bo) - sh), (float)cnt);
        }
      }
      __syncthreads();
    }
    if (PRE) {
      const int q = zin - 2 * kNu - 1;
      if (q >= z0 && q < z1) {
        const float* xp = xs + (q % G::RX) * G::P;
        const float* xm = xs + ((q + G::RX - 1) % G::RX) * G::P;
        const float* xq = xs + ((q + 1) % G::RX) * G::P;
        const bool hm = q > 0, hq = q < n - 1;
        float* out = xout + (int64_t)q * nn;
        const float* bq = b + (int64_t)q * nn;
        for (int c = threadIdx.x; c < kTX * kTY; c += blockDim.x) {
          const int gx = X0 + c % kTX, gy = Y0 + c / kTX;
          if (gx < n && gy < n) out[gy * n + gx] = xp[(gy - Y0 + G::H) * G::WX + (gx - X0 + G::H)];
        }
        // one thread per coarse cell of this plane: residual of its 4 children, fixed order
        for (int c = threadIdx.x; c < (kTX / 2) * (kTY / 2); c += blockDim.x) {
          const int cx = c % (kTX / 2), cy = c / (kTX / 2);
          float r = 0.f;
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            const int gx = X0 + 2 * cx + (ch & 1), gy = Y0 + 2 * cy + (ch >> 1);
            if (gx >= n || gy >= n) continue;
            const int lc = (gy - Y0 + G::H) * G::WX + (gx - X0 + G::H);
            const float xv = xp[lc];
            float lx = 0.f;
            if (gx > 0) lx += xp[lc - 1] - xv;
            if (gx < n - 1) lx += xp[lc + 1] - xv;
            if (gy > 0) lx += xp[lc - G::WX] - xv;
            if (gy < n - 1) lx += xp[lc + G::WX] - xv;
            if (hm) lx += xm[lc] - xv;
            if (hq) lx += xq[lc] - xv;
            r += (__ldg(bq + gy * n + gx) - sh) - lx;
          }
          if ((q & 1) == 0) {
            cacc[c] = r;
          } else {
            const int gcx = (X0 >> 1) + cx, gcy = (Y0 >> 1) + cy;
            if (gcx < nc && gcy < nc) bc[lin(gcx, gcy, q >> 1, nc)] = 0.5f * (cacc[c] + r);
          }
        }
      }
      __syncthreads();
    } else {
      const int p = zin - 2 * kNu;
      if (p >= z0 && p < z1) {
        const float* xp = xs + (p % G::RX) * G::P;
        float* out = xout + (int64_t)p * nn;
        for (int c = threadIdx.x; c < kTX * kTY; c += blockDim.x) {
          const int gx = X0 + c % kTX, gy = Y0 + c / kTX;
          if (gx < n && gy < n) out[gy * n + gx] = xp[(gy - Y0 + G::H) * G::WX + (gx - X0 + G::H)];
        }
      }
      __syncthreads();
    }
  }
}


// ---------------------------------------------------------------- mid-size levels
// 16 < n < kFusedMin: one launch per half-sweep (launch-latency regime, the
// level is L2-resident).  In place on x.
__global__ void zero_kernel(float* __restrict__ x, int64_t N, const int* __restrict__ gate) {
  if (*gate) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] = 0.f;
}

__global__ void rbgs_kernel(float* __restrict__ x, const float* __restrict__ b,
                            const double* __restrict__ shift, int n, int color,
                            const int* __restrict__ gate) {
  if (*gate) return;
  const int half = n >> 1;
  const int64_t M = (int64_t)half * n * n;
  const float sh = shift ? (float)*shift : 0.f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int ih = (int)(t % half);
    const int64_t row = t / half;
    const int j = (int)(row % n), k = (int)(row / n);
    const int i = 2 * ih + ((j + k + color) & 1);
    const int64_t p = lin(i, j, k, n);
    float s = 0.f;
    int cnt = 0;
    if (i > 0) { s += x[p - 1]; ++cnt; }
    if (i < n - 1) { s += x[p + 1]; ++cnt; }
    if (j > 0) { s += x[p - n]; ++cnt; }
    if (j < n - 1) { s += x[p + n]; ++cnt; }
    if (k > 0) { s += x[p - (int64_t)n * n]; ++cnt; }
    if (k < n - 1) { s += x[p + (int64_t)n * n]; ++cnt; }
    x[p] = (s - (b[p] - sh)) / (float)cnt;
  }
}

__global__ void resid_restrict_kernel(const float* __restrict__ x, const float* __restrict__ b,
                                      const double* __restrict__ shift, int n,
                                      float* __restrict__ bc, const int* __restrict__ gate) {
  if (*gate) return;
  const int nc = n >> 1;
  const int64_t Mc = (int64_t)nc * nc * nc;
  const float sh = shift ? (float)*shift : 0.f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < Mc;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(t % nc), J = (int)((t / nc) % nc), K = (int)(t / ((int64_t)nc * nc));
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
      const int64_t p = lin(i, j, k, n);
      const float xc = x[p];
      float lx = 0.f;
      if (i > 0) lx += x[p - 1] - xc;
      if (i < n - 1) lx += x[p + 1] - xc;
      if (j > 0) lx += x[p - n] - xc;
      if (j < n - 1) lx += x[p + n] - xc;
      if (k > 0) lx += x[p - (int64_t)n * n] - xc;
      if (k < n - 1) lx += x[p + (int64_t)n * n] - xc;
      acc += (b[p] - sh) - lx;
    }
    bc[t] = 0.5f * acc;
  }
}

__global__ void prolong_kernel(const float* __restrict__ xc, float* __restrict__ x, int n,
                               const int* __restrict__ gate) {
  if (*gate) return;
  const int nc = n >> 1;
  const int64_t N = (int64_t)n * n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
    x[t] += prolong_at(xc, nc, i, j, k);
  }
}


// ---------------------------------------------------------------- small grids
// A whole V-cycle hierarchy for n <= 16 in one CTA's shared memory: solves
// L x = b - shift - mean approximately (2 V-cycles from zero), writes x.
constexpr int kSmallCap = 4096 + 512 + 64 + 27 + 8;

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
                                                            const double* __restrict__ shift, int n0,
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
  const float sh = shift ? (float)*shift : 0.f;
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
  for (int cyc = 0; cyc < 2; ++cyc) {
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
      const int sweeps = 2 * n * n + 16;
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

__global__ void rhs_stats64_kernel(const double* __restrict__ b, int64_t N,
                                   double* __restrict__ partials) {
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[t];
    s1 += v;
    s2 += v * v;
  }
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
    ss->bnorm = sqrt(fmax(s2 - s1 * mean, 0.0));
  }
}

// One V-cycle on level l.  x0 / x0b: level-0 iterate and its ping-pong
// partner; b0, shift0: level-0 right-hand side.  zero0: level-0 x is zero.
int vcycle(wgeo_handle* h, int l, float* x0, float* x0b, const float* b0, const double* shift0, bool zero0,
           const int* gate, cudaStream_t s) {
  const int n = h->levels[l].n;
  float* x = (l == 0) ? x0 : h->levels[l].x;
  float* xb = (l == 0) ? x0b : h->levels[l].x2;
  const float* b = (l == 0) ? b0 : h->levels[l].b;
  const double* shift = (l == 0) ? shift0 : nullptr;
  if (n <= kSmallN || l == h->nlevels - 1) {
    small_vcycle_kernel<<<1, 1024, 0, s>>>(x, b, shift, n, gate);
    WGEO_LAUNCH_CHECK();
    return WGEO_OK;
  }
  const bool zero = (l == 0) ? zero0 : true;
  const int nc = n >> 1;
  const int64_t N = (int64_t)n * n * n, Nc = (int64_t)nc * nc * nc;
  if (n < kFusedMin) {
    // mid-size level: in place, one launch per half-sweep
    const int gb = grid_blocks(N / 2, kThreads, 152 * 32);
    if (zero) {
      zero_kernel<<<grid_blocks(N, kThreads, 152 * 32), kThreads, 0, s>>>(x, N, gate);
      WGEO_LAUNCH_CHECK();
    }
    for (int sw = 0; sw < kNu; ++sw)
      for (int c = 0; c < 2; ++c) {
        rbgs_kernel<<<gb, kThreads, 0, s>>>(x, b, shift, n, c, gate);
        WGEO_LAUNCH_CHECK();
      }
    resid_restrict_kernel<<<grid_blocks(Nc, kThreads, 152 * 32), kThreads, 0, s>>>(x, b, shift, n,
                                                                                  h->levels[l + 1].b, gate);
    WGEO_LAUNCH_CHECK();
    int rc = vcycle(h, l + 1, x0, x0b, b0, shift0, zero0, gate, s);
    if (rc) return rc;
    prolong_kernel<<<grid_blocks(N, kThreads, 152 * 32), kThreads, 0, s>>>(h->levels[l + 1].x, x, n, gate);
    WGEO_LAUNCH_CHECK();
    for (int sw = 0; sw < kNu; ++sw)
      for (int c = 1; c >= 0; --c) {
        rbgs_kernel<<<gb, kThreads, 0, s>>>(x, b, shift, n, c, gate);
        WGEO_LAUNCH_CHECK();
      }
    return WGEO_OK;
  }
  // z chunk: a CTA's pipeline costs ~ (zc + 3 * 2 kNu) plane steps and runs in
  // ceil(CTAs / resident CTAs) waves; take the chunk with the lowest product
  int zc = 16;
  {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int slots = 2 * sms;
    long best = -1;
    for (int cand = 16; cand <= 64; cand *= 2) {
      const long ctas = (long)div_up(n, kTX) * div_up(n, kTY) * div_up(n, cand);
      const long cost = ((ctas + slots - 1) / slots) * (cand + 6 * kNu);
      if (best < 0 || cost < best) {
        best = cost;
        zc = cand;
      }
    }
  }
  const dim3 grid(div_up(n, kTX), div_up(n, kTY), div_up(n, zc));
  if (zero)
    smooth_kernel<true, true><<<grid, kSmThreads, SmGeom<true>::smem, s>>>(x, xb, b, shift, n, zc, nullptr,
                                                                           h->levels[l + 1].b, gate);
  else
    smooth_kernel<true, false><<<grid, kSmThreads, SmGeom<true>::smem, s>>>(x, xb, b, shift, n, zc, nullptr,
                                                                            h->levels[l + 1].b, gate);
  WGEO_LAUNCH_CHECK();
  int rc = vcycle(h, l + 1, x0, x0b, b0, shift0, zero0, gate, s);
  if (rc) return rc;
  smooth_kernel<false, false><<<grid, kSmThreads, SmGeom<false>::smem, s>>>(xb, x, b, shift, n, zc,
                                                                            h->levels[l + 1].x, nullptr, gate);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

// The fixed launch sequence of one solve (mode 0: forward, 1: adjoint).
int enqueue_solve(wgeo_handle* h, int res, int mode, cudaStream_t s) {
  const int64_t N = (int64_t)res * res * res;
  SolveState* ss = mode == 0 ? &h->dstate->fwd : &h->dstate->bwd;
  const int* gate = &ss->done;
  const bool fp32 = (mode == 0 && h->opt.precision == WGEO_PREC_FP32);
  const int rb = grid_blocks(N, kThreads, kPartials);
  if (fp32) {
    const double tol = h->opt.tol_rel;
    const int maxv = h->opt.max_vcycles;
    for (int it = 0; it <= maxv; ++it) {
      residual32_kernel<<<rb, kThreads, 0, s>>>(h->chi32, h->b32, &ss->bmean, res, h->partials, gate);
      WGEO_LAUNCH_CHECK();
      finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss, h->dstate, tol, it, it == maxv, 1, 0);
      WGEO_LAUNCH_CHECK();
      if (it == maxv) break;
      int rc = vcycle(h, 0, h->chi32, h->r32, h->b32, &ss->bmean, false, gate, s);
      if (rc) return rc;
    }
    return WGEO_OK;
  }
  const double tol = mode == 0 ? h->opt.tol_rel : h->opt.tol_rel_adjoint;
  PairFF xp;
  xp.buf[0] = mode == 0 ? h->chiff[0] : h->lamff[0];
  xp.buf[1] = mode == 0 ? h->chiff[1] : h->lamff[1];
  float* x32 = mode == 0 ? h->chi32 : h->lam32;
  const int maxr = h->opt.max_refine;
  const int nv = h->opt.vcycles_per_refine;
  for (int it = 0; it <= maxr; ++it) {
    const float* e = it == 0 ? nullptr : h->e32;
    if (mode == 0)
      update_residual_kernel<float><<<rb, kThreads, 0, s>>>(xp, e, h->b32, res, h->r32, x32, h->partials, ss);
    else
      update_residual_kernel<double><<<rb, kThreads, 0, s>>>(xp, e, h->dchi64, res, h->r32, x32, h->partials, ss);
    WGEO_LAUNCH_CHECK();
    finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss, h->dstate, tol, it, it == maxr, 0, e ? 1 : 0);
    WGEO_LAUNCH_CHECK();
    if (it == maxr) break;
    // correction: V-cycles on L e = r - mean(r); the FP32 copy x32 serves as the
    // ping-pong partner (it is rewritten by the next refinement pass)
    for (int v = 0; v < nv; ++v) {
      int rc = vcycle(h, 0, h->e32, x32, h->r32, &ss->rmean, v == 0, gate, s);
      if (rc) return rc;
    }
  }
  return WGEO_OK;
}

}  // namespace

int coarsest_size(int res) {
  int n = res;
  while ((n % 2) == 0 && n > 8) n /= 2;
  return n;
}

int build_levels(wgeo_handle* h, int res) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(smooth_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SmGeom<true>::smem);
    cudaFuncSetAttribute(smooth_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SmGeom<true>::smem);
    cudaFuncSetAttribute(smooth_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SmGeom<false>::smem);
    attr_done = true;
  }
  int n = res;
  int l = 0;
  float* pool = h->level_pool;
  h->levels[0].n = n;
  h->levels[0].x = nullptr;
  h->levels[0].x2 = nullptr;
  h->levels[0].b = nullptr;
  while ((n % 2) == 0 && n > 8) {
    n /= 2;
    ++l;
    if (l >= kMaxLevels) return WGEO_ERR_INVALID_ARG;
    const int64_t M = (int64_t)n * n * n;
    const int64_t Ma = (M + 63) / 64 * 64;
    h->levels[l].n = n;
    h->levels[l].x = pool;
    h->levels[l].x2 = pool + Ma;
    h->levels[l].b = pool + 2 * Ma;
    pool += 3 * Ma;
  }
  if (n > 16) return WGEO_ERR_INVALID_ARG;
  h->nlevels = l + 1;
  return WGEO_OK;
}

// Enqueues one solve.  The launch sequence depends only on (res, mode,
// options), and every pointer it uses is owned by the handle, so it is
// recorded once as a CUDA graph and replayed; while the caller's stream is
// itself being captured the kernels are enqueued directly instead.
int launch_solve(wgeo_handle* h, int res, int mode, bool cold, cudaStream_t s) {
  const int64_t N = (int64_t)res * res * res;
  SolveState* ss = mode == 0 ? &h->dstate->fwd : &h->dstate->bwd;
  if (mode == 1) {
    const int rb = grid_blocks(N, kThreads, kPartials);
    rhs_stats64_kernel<<<rb, kThreads, 0, s>>>(h->dchi64, N, h->partials);
    WGEO_LAUNCH_CHECK();
    rhs_stats_finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss);
    WGEO_LAUNCH_CHECK();
  }
  solve_begin_kernel<<<1, 1, 0, s>>>(ss, cold ? 1 : 0);
  WGEO_LAUNCH_CHECK();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  WGEO_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (!h->opt.use_graphs || cap != cudaStreamCaptureStatusNone) return enqueue_solve(h, res, mode, s);
  SolverGraph& g = h->graphs[mode];
  const int gmode = mode * 2 + (h->opt.precision == WGEO_PREC_FP32 ? 1 : 0);
  if (g.exec == nullptr || g.res != res || g.mode != gmode) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (!h->capture_stream) WGEO_CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    WGEO_CUDA_TRY(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    const long long before = t_kernel_launches;
    int rc = enqueue_solve(h, res, mode, h->capture_stream);
    // recorded, not run: counted at each replay instead
    const long long captured = t_kernel_launches - before;
    t_kernel_launches -= captured;
    g_kernel_launches.fetch_sub(captured, std::memory_order_relaxed);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->capture_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return WGEO_ERR_CUDA;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return WGEO_ERR_CUDA;
    }
    g.res = res;
    g.mode = gmode;
    g.launches = captured;
  }
  WGEO_CUDA_TRY(cudaGraphLaunch(g.exec, s));
  g_kernel_launches.fetch_add(g.launches, std::memory_order_relaxed);
  t_kernel_launches += g.launches;
  return WGEO_OK;
}

}  // namespace wgeo
