// Poisson solve A a = b (Sec. 2.3, Eqs. 15, 20-21; adjoint solve Eq. 38).
//
// Operator: unit-free cell-centred 7-point Neumann Laplacian
//   (L x)_p = sum over in-grid neighbours q of (x_q - x_p),
// the transverse-lumped trilinear Galerkin stiffness (up to sign and a factor
// h).  The system is singular (constants) and consistent after projecting the
// mean out of the right-hand side; chi is defined up to an additive constant.
//
// Mixed precision (default): FP64 iterative refinement around FP32 multigrid.
//   r = b - L x64 in FP64 (block partial sums of r and r^2 in FP64, reduced in
//   a fixed order), convergence test ||r - mean r|| <= tol ||b - mean b||,
//   then V-cycles in FP32 on L e = r - mean(r), x64 += e.
// Plain FP32 (comparator): V-cycles directly on x32 with an FP32 residual.
//
// Multigrid: cell-centred, halving while the grid is even and larger than 8;
// red-black Gauss-Seidel (2 pre, 2 post sweeps), residual restricted by
// summing the 8 children with weight 1/2 (average times H^2/h^2 = 4 for the
// unit-free operator), trilinear prolongation with mirrored Neumann edges,
// coarsest grid (<= 16^3) solved by Gauss-Seidel sweeps in one CTA.
//
// Every kernel after the first convergence test reads the solve's `done` flag
// and returns at once when it is set, so the fixed launch sequence (recorded
// once as a CUDA graph) stops doing work as soon as the tolerance is met.
#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

constexpr int kThreads = 256;
constexpr int kNu1 = 2, kNu2 = 2;

__device__ __forceinline__ int64_t lin(int i, int j, int k, int n) {
  return ((int64_t)k * n + j) * n + i;
}

template <typename TB>
__global__ void residual64_kernel(const double* __restrict__ x, const TB* __restrict__ b, int n,
                                  float* __restrict__ r32, double* __restrict__ partials,
                                  const int* __restrict__ gate) {
  if (*gate) return;
  __shared__ double red[32];
  const int64_t N = (int64_t)n * n * n;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
    const double xc = x[t];
    double acc = 0.0;
    if (i > 0) acc += x[t - 1] - xc;
    if (i < n - 1) acc += x[t + 1] - xc;
    if (j > 0) acc += x[t - n] - xc;
    if (j < n - 1) acc += x[t + n] - xc;
    if (k > 0) acc += x[t - (int64_t)n * n] - xc;
    if (k < n - 1) acc += x[t + (int64_t)n * n] - xc;
    const double r = (double)b[t] - acc;
    r32[t] = (float)r;
    s1 += r;
    s2 += r * r;
  }
  s1 = block_sum<kThreads>(s1, red);
  s2 = block_sum<kThreads>(s2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1;
    partials[2 * blockIdx.x + 1] = s2;
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
  if (l == 0) {
    red[w] = s1;
  }
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
// fp32 != 0: sums in float (the plain FP32 comparator's dots).
__global__ void finalize_kernel(const double* __restrict__ partials, int nblocks, int64_t N,
                                SolveState* ss, DevState* st, double tol, int step, int last,
                                int fp32) {
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

__global__ void solve_begin_kernel(SolveState* ss) {
  ss->done = 0;
  ss->iter = 0;
  ss->rel = 0.0;
  ss->rmean = 0.0;
}

__global__ void zero_kernel(float* __restrict__ x, int64_t N, const int* __restrict__ gate) {
  if (*gate) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] = 0.f;
}

// One colour of red-black Gauss-Seidel; colour of (i,j,k) is (i+j+k) & 1.
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

// bc(I,J,K) = 1/2 * sum over the 8 children of (b - shift - L x).
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

// x_fine += P x_coarse (trilinear between coarse cell centres, 3/4-1/4 per axis,
// the outside neighbour mirrored onto the edge cell).
__global__ void prolong_kernel(const float* __restrict__ xc, float* __restrict__ x, int n,
                               const int* __restrict__ gate) {
  if (*gate) return;
  const int nc = n >> 1;
  const int64_t N = (int64_t)n * n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    int I2 = (i & 1) ? I + 1 : I - 1;
    int J2 = (j & 1) ? J + 1 : J - 1;
    int K2 = (k & 1) ? K + 1 : K - 1;
    I2 = min(max(I2, 0), nc - 1);
    J2 = min(max(J2, 0), nc - 1);
    K2 = min(max(K2, 0), nc - 1);
    const float a = 0.75f, c = 0.25f;
    const float v =
        a * a * a * xc[lin(I, J, K, nc)] + c * a * a * xc[lin(I2, J, K, nc)] +
        a * c * a * xc[lin(I, J2, K, nc)] + a * a * c * xc[lin(I, J, K2, nc)] +
        c * c * a * xc[lin(I2, J2, K, nc)] + c * a * c * xc[lin(I2, J, K2, nc)] +
        a * c * c * xc[lin(I, J2, K2, nc)] + c * c * c * xc[lin(I2, J2, K2, nc)];
    x[t] += v;
  }
}

// Coarsest grid (n^3 <= 4096): mean-projected right-hand side, Gauss-Seidel
// sweeps in shared memory by one CTA.
__global__ void __launch_bounds__(1024) coarse_kernel(float* __restrict__ x,
                                                      const float* __restrict__ b,
                                                      const double* __restrict__ shift, int n,
                                                      int sweeps, const int* __restrict__ gate) {
  if (*gate) return;
  __shared__ float xs[4096];
  __shared__ float bs[4096];
  __shared__ double red[32];
  const int N = n * n * n;
  const float sh = shift ? (float)*shift : 0.f;
  double s = 0.0;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    bs[t] = b[t] - sh;
    xs[t] = 0.f;
    s += bs[t];
  }
  s = block_sum<1024>(s, red);
  __shared__ float meanb;
  if (threadIdx.x == 0) meanb = (float)(s / N);
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) bs[t] -= meanb;
  __syncthreads();
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int color = 0; color < 2; ++color) {
      for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, k = t / (n * n);
        if (((i + j + k) & 1) != color) continue;
        float acc = 0.f;
        int cnt = 0;
        if (i > 0) { acc += xs[t - 1]; ++cnt; }
        if (i < n - 1) { acc += xs[t + 1]; ++cnt; }
        if (j > 0) { acc += xs[t - n]; ++cnt; }
        if (j < n - 1) { acc += xs[t + n]; ++cnt; }
        if (k > 0) { acc += xs[t - n * n]; ++cnt; }
        if (k < n - 1) { acc += xs[t + n * n]; ++cnt; }
        xs[t] = cnt ? (acc - bs[t]) / (float)cnt : 0.f;
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < N; t += blockDim.x) x[t] = xs[t];
}

__global__ void update64_kernel(double* __restrict__ x64, const float* __restrict__ e, int64_t N,
                                const int* __restrict__ gate) {
  if (*gate) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    x64[t] += (double)e[t];
}

__global__ void to_f32_kernel(const double* __restrict__ x64, float* __restrict__ x32, int64_t N) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    x32[t] = (float)x64[t];
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

int coarse_sweeps(int n) { return 2 * n * n + 16; }

int vcycle(wgeo_handle* h, int l, float* x0, const float* b0, const double* shift0,
           const int* gate, cudaStream_t s) {
  const int n = h->levels[l].n;
  float* x = (l == 0) ? x0 : h->levels[l].x;
  const float* b = (l == 0) ? b0 : h->levels[l].b;
  const double* shift = (l == 0) ? shift0 : nullptr;
  if (l == h->nlevels - 1) {
    coarse_kernel<<<1, 1024, 0, s>>>(x, b, shift, n, coarse_sweeps(n), gate);
    WGEO_LAUNCH_CHECK();
    return WGEO_OK;
  }
  const int64_t N = (int64_t)n * n * n;
  const int gb = grid_blocks(N / 2, kThreads, 152 * 32);
  for (int sw = 0; sw < kNu1; ++sw)
    for (int c = 0; c < 2; ++c) {
      rbgs_kernel<<<gb, kThreads, 0, s>>>(x, b, shift, n, c, gate);
      WGEO_LAUNCH_CHECK();
    }
  const int nc = n >> 1;
  const int64_t Nc = (int64_t)nc * nc * nc;
  resid_restrict_kernel<<<grid_blocks(Nc, kThreads, 152 * 32), kThreads, 0, s>>>(
      x, b, shift, n, h->levels[l + 1].b, gate);
  WGEO_LAUNCH_CHECK();
  if (l + 1 != h->nlevels - 1) {
    zero_kernel<<<grid_blocks(Nc, kThreads, 152 * 32), kThreads, 0, s>>>(h->levels[l + 1].x, Nc, gate);
    WGEO_LAUNCH_CHECK();
  }
  int rc = vcycle(h, l + 1, x0, b0, shift0, gate, s);
  if (rc) return rc;
  prolong_kernel<<<grid_blocks(N, kThreads, 152 * 32), kThreads, 0, s>>>(h->levels[l + 1].x, x, n, gate);
  WGEO_LAUNCH_CHECK();
  for (int sw = 0; sw < kNu2; ++sw)
    for (int c = 1; c >= 0; --c) {
      rbgs_kernel<<<gb, kThreads, 0, s>>>(x, b, shift, n, c, gate);
      WGEO_LAUNCH_CHECK();
    }
  return WGEO_OK;
}

// The fixed launch sequence of one solve (mode 0: forward, 1: adjoint).
int enqueue_solve(wgeo_handle* h, int res, int mode, cudaStream_t s) {
  const int64_t N = (int64_t)res * res * res;
  SolveState* ss = mode == 0 ? &h->dstate->fwd : &h->dstate->bwd;
  const int* gate = &ss->done;
  const bool fp32 = (mode == 0 && h->opt.precision == WGEO_PREC_FP32);
  const int rb = grid_blocks(N, kThreads, kPartials);
  const double tol = h->opt.tol_rel;
  solve_begin_kernel<<<1, 1, 0, s>>>(ss);
  WGEO_LAUNCH_CHECK();
  if (fp32) {
    const int maxv = h->opt.max_vcycles;
    for (int it = 0; it <= maxv; ++it) {
      residual32_kernel<<<rb, kThreads, 0, s>>>(h->chi32, h->b32, &ss->bmean, res, h->partials, gate);
      WGEO_LAUNCH_CHECK();
      finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss, h->dstate, tol, it, it == maxv, 1);
      WGEO_LAUNCH_CHECK();
      if (it == maxv) break;
      int rc = vcycle(h, 0, h->chi32, h->b32, &ss->bmean, gate, s);
      if (rc) return rc;
    }
    return WGEO_OK;
  }
  double* x64 = mode == 0 ? h->chi64 : h->lam64;
  float* x32 = mode == 0 ? h->chi32 : h->lam32;
  const int maxr = h->opt.max_refine;
  const int nv = h->opt.vcycles_per_refine;
  for (int it = 0; it <= maxr; ++it) {
    if (mode == 0)
      residual64_kernel<float><<<rb, kThreads, 0, s>>>(x64, h->b32, res, h->r32, h->partials, gate);
    else
      residual64_kernel<double><<<rb, kThreads, 0, s>>>(x64, h->dchi64, res, h->r32, h->partials, gate);
    WGEO_LAUNCH_CHECK();
    finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, ss, h->dstate, tol, it, it == maxr, 0);
    WGEO_LAUNCH_CHECK();
    if (it == maxr) break;
    zero_kernel<<<grid_blocks(N, kThreads, 152 * 32), kThreads, 0, s>>>(h->e32, N, gate);
    WGEO_LAUNCH_CHECK();
    for (int v = 0; v < nv; ++v) {
      int rc = vcycle(h, 0, h->e32, h->r32, &ss->rmean, gate, s);
      if (rc) return rc;
    }
    update64_kernel<<<grid_blocks(N, kThreads, 152 * 32), kThreads, 0, s>>>(x64, h->e32, N, gate);
    WGEO_LAUNCH_CHECK();
  }
  to_f32_kernel<<<grid_blocks(N, kThreads, 152 * 32), kThreads, 0, s>>>(x64, x32, N);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

}  // namespace

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
  while ((n % 2) == 0 && n > 8) {
    n /= 2;
    ++l;
    if (l >= kMaxLevels) return WGEO_ERR_INVALID_ARG;
    const int64_t M = (int64_t)n * n * n;
    h->levels[l].n = n;
    h->levels[l].x = pool;
    pool += (M + 63) / 64 * 64;
    h->levels[l].b = pool;
    pool += (M + 63) / 64 * 64;
  }
  if (n > 16) return WGEO_ERR_INVALID_ARG;
  h->nlevels = l + 1;
  return WGEO_OK;
}

// Enqueues one solve.  The launch sequence depends only on (res, mode,
// options), and every pointer it uses is owned by the handle, so it is
// recorded once as a CUDA graph and replayed; while the caller's stream is
// itself being captured the kernels are enqueued directly instead.
int launch_solve(wgeo_handle* h, int res, int mode, cudaStream_t s) {
  const int64_t N = (int64_t)res * res * res;
  if (mode == 1) {
    const int rb = grid_blocks(N, kThreads, kPartials);
    rhs_stats64_kernel<<<rb, kThreads, 0, s>>>(h->dchi64, N, h->partials);
    WGEO_LAUNCH_CHECK();
    rhs_stats_finalize_kernel<<<1, 1024, 0, s>>>(h->partials, rb, N, &h->dstate->bwd);
    WGEO_LAUNCH_CHECK();
  }
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
    int rc = enqueue_solve(h, res, mode, h->capture_stream);
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
  }
  WGEO_CUDA_TRY(cudaGraphLaunch(g.exec, s));
  return WGEO_OK;
}

}  // namespace wgeo
