// Differentiable shape parameterisation (Sec. 2.5 last paragraph, Sec. 3.3):
// a star body r(u) = base + sum_k theta_k Y_k(u) with orthonormal real
// spherical harmonics (no Condon-Shortley phase, k = l*l + l + m), sampled at
// fixed unit directions u_i:  x_i = centre + r(u_i) u_i and the outward normal
// n_i = m_i / |m_i|, m_i = u_i - P_perp grad r / r.
//
// SH are evaluated in Cartesian form: Y_lm = sqrt(2) K_lm Q_l^m(z) Re/Im (x+iy)^m
// (K_l0 Q_l^0 for m = 0) with Q_l^m the polynomial part of P_l^m, so the
// Cartesian gradient of the polynomial extension has no pole singularity.
//
// The adjoint reduces sum_i over points per coefficient with warp shuffles,
// per-warp shared slots and a fixed-order final pass (deterministic).
#include <math.h>

#include <mutex>

#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

constexpr int kLmax = 8;
constexpr int kK = (kLmax + 1) * (kLmax + 1);
constexpr int kShThreads = 128;
constexpr int kShBlocks = 256;

struct ShConsts {
  double K[kLmax + 1][kLmax + 1];  // K_lm
  int lmax;
};

// Y_k and the Cartesian gradient of the polynomial extension, for all k.
__device__ __forceinline__ void eval_sh(const float u[3], const ShConsts& cs, float* Y, float (*dY)[3]) {
  // recurrences in FP64 (the three-term Legendre recurrence cancels), stored as float
  const double x = u[0], y = u[1], z = u[2];
  double C[kLmax + 1], S[kLmax + 1];
  C[0] = 1.0;
  S[0] = 0.0;
  for (int m = 1; m <= cs.lmax; ++m) {
    C[m] = x * C[m - 1] - y * S[m - 1];
    S[m] = x * S[m - 1] + y * C[m - 1];
  }
  for (int m = 0; m <= cs.lmax; ++m) {
    double dfact = 1.0;
    for (int j = 1; j < 2 * m; j += 2) dfact *= (double)j;
    double q2 = 0.0, dq2 = 0.0;         // Q_{l-2}
    double q1 = dfact, dq1 = 0.0;       // Q_{l-1} (starts at l = m)
    for (int l = m; l <= cs.lmax; ++l) {
      double q, dq;
      if (l == m) {
        q = dfact;
        dq = 0.0;
      } else if (l == m + 1) {
        q = (2 * m + 1) * z * q1;
        dq = (2 * m + 1) * (q1 + z * dq1);
      } else {
        q = ((2 * l - 1) * z * q1 - (l + m - 1) * q2) / (double)(l - m);
        dq = ((2 * l - 1) * (q1 + z * dq1) - (l + m - 1) * dq2) / (double)(l - m);
      }
      if (l > m) {
        q2 = q1;
        dq2 = dq1;
        q1 = q;
        dq1 = dq;
      }
      const double K = cs.K[l][m];
      if (m == 0) {
        const int k = l * l + l;
        Y[k] = (float)(K * q);
        dY[k][0] = 0.f;
        dY[k][1] = 0.f;
        dY[k][2] = (float)(K * dq);
      } else {
        const double s2 = 1.4142135623730951 * K;
        const int kc = l * l + l + m, ks = l * l + l - m;
        Y[kc] = (float)(s2 * q * C[m]);
        Y[ks] = (float)(s2 * q * S[m]);
        dY[kc][0] = (float)(s2 * q * m * C[m - 1]);
        dY[kc][1] = (float)(-s2 * q * m * S[m - 1]);
        dY[kc][2] = (float)(s2 * dq * C[m]);
        dY[ks][0] = (float)(s2 * q * m * S[m - 1]);
        dY[ks][1] = (float)(s2 * q * m * C[m - 1]);
        dY[ks][2] = (float)(s2 * dq * S[m]);
      }
    }
  }
}

struct Surf {
  float r;
  float gt[3];  // tangential gradient of r
  float m[3];
  float mn;     // |m|
  float n[3];
};

__device__ __forceinline__ Surf surface_at(const float u[3], const float* __restrict__ theta, int K,
                                           float base, const float* Y, const float (*dY)[3]) {
  // r and grad r accumulate up to 81 terms with |grad Y| ~ 20 and cancellation:
  // FP64 here keeps the normals at float32 accuracy
  Surf s;
  double r = base, g[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k) {
    const double t = theta[k];
    r += t * Y[k];
    g[0] += t * dY[k][0];
    g[1] += t * dY[k][1];
    g[2] += t * dY[k][2];
  }
  const double gu = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];
  double m[3];
  for (int a = 0; a < 3; ++a) {
    const double gt = g[a] - gu * u[a];
    s.gt[a] = (float)gt;
    m[a] = u[a] - gt / r;
  }
  const double mn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  for (int a = 0; a < 3; ++a) {
    s.m[a] = (float)m[a];
    s.n[a] = (float)(m[a] / mn);
  }
  s.mn = (float)mn;
  s.r = (float)r;
  return s;
}

__global__ void sh_surface_kernel(const float* __restrict__ theta, int K, ShConsts cs,
                                  const float* __restrict__ dirs, int64_t n, float base,
                                  const float* __restrict__ centre, float* __restrict__ pts,
                                  float* __restrict__ nrm) {
  float Y[kK], dY[kK][3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float u[3] = {dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
    eval_sh(u, cs, Y, dY);
    const Surf s = surface_at(u, theta, K, base, Y, dY);
    for (int a = 0; a < 3; ++a) {
      pts[3 * i + a] = centre[a] + s.r * u[a];
      nrm[3 * i + a] = s.n[a];
    }
  }
}

__global__ void __launch_bounds__(kShThreads) sh_backward_kernel(
    const float* __restrict__ theta, int K, ShConsts cs, const float* __restrict__ dirs, int64_t n,
    float base, const float* __restrict__ dpts, const float* __restrict__ dnrm,
    double* __restrict__ partials) {
  __shared__ double acc[kK][kShThreads / 32];
  for (int t = threadIdx.x; t < kK * (kShThreads / 32); t += blockDim.x) (&acc[0][0])[t] = 0.0;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float Y[kK], dY[kK][3];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (n + stride - 1) / stride;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t i = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool act = i < n;
    float A = 0.f, B[3] = {0.f, 0.f, 0.f}, Cc = 0.f, u[3] = {0.f, 0.f, 1.f};
    if (act) {
      u[0] = dirs[3 * i];
      u[1] = dirs[3 * i + 1];
      u[2] = dirs[3 * i + 2];
      eval_sh(u, cs, Y, dY);
      const Surf s = surface_at(u, theta, K, base, Y, dY);
      const float dp[3] = {dpts[3 * i], dpts[3 * i + 1], dpts[3 * i + 2]};
      const float dn[3] = {dnrm[3 * i], dnrm[3 * i + 1], dnrm[3 * i + 2]};
      A = dp[0] * u[0] + dp[1] * u[1] + dp[2] * u[2];
      const float pr = s.n[0] * dn[0] + s.n[1] * dn[1] + s.n[2] * dn[2];
      float dm[3];
      for (int a = 0; a < 3; ++a) dm[a] = (dn[a] - s.n[a] * pr) / s.mn;
      for (int a = 0; a < 3; ++a) B[a] = dm[a] / s.r;
      Cc = (dm[0] * s.gt[0] + dm[1] * s.gt[1] + dm[2] * s.gt[2]) / (s.r * s.r);
    }
    const float uB = u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
    for (int k = 0; k < K; ++k) {
      double v = 0.0;
      if (act) {
        const float dyb = dY[k][0] * B[0] + dY[k][1] * B[1] + dY[k][2] * B[2];
        const float dyu = dY[k][0] * u[0] + dY[k][1] * u[1] + dY[k][2] * u[2];
        v = (double)(Y[k] * (A + Cc)) - (double)(dyb - dyu * uB);
      }
      v = warp_sum(v);
      if (lane == 0) acc[k][w] += v;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kShThreads / 32; ++q) s += acc[k][q];
    partials[(int64_t)blockIdx.x * K + k] = s;
  }
}

__global__ void sh_finalize_kernel(const double* __restrict__ partials, int nblocks, int K,
                                   float* __restrict__ dtheta) {
  const int k = threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * K + k];
  dtheta[k] = (float)s;
}

ShConsts make_consts(int K) {
  ShConsts cs;
  cs.lmax = (int)lround(sqrt((double)K)) - 1;
  for (int l = 0; l <= kLmax; ++l)
    for (int m = 0; m <= kLmax; ++m) {
      if (m > l) {
        cs.K[l][m] = 0.0;
        continue;
      }
      double r = 1.0;
      for (int j = l - m + 1; j <= l + m; ++j) r /= (double)j;   // (l-m)!/(l+m)!
      cs.K[l][m] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * r);
    }
  return cs;
}

}  // namespace

int launch_sh_surface(const float* theta, int K, const float* dirs, int64_t n, float base,
                      const float* centre, float* points, float* normals, cudaStream_t s) {
  if (n == 0) return WGEO_OK;
  sh_surface_kernel<<<grid_blocks(n, 128, 152 * 16), 128, 0, s>>>(theta, K, make_consts(K), dirs, n, base,
                                                                 centre, points, normals);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

int launch_sh_backward(wgeo_handle* h, const float* theta, int K, const float* dirs, int64_t n,
                       float base, const float* dpts, const float* dnrm, float* dtheta, cudaStream_t s) {
  const int nb = (n == 0) ? 1 : grid_blocks(n, kShThreads, kShBlocks);
  if (n == 0) {
    WGEO_CUDA_TRY(cudaMemsetAsync(dtheta, 0, sizeof(float) * K, s));
    return WGEO_OK;
  }
  sh_backward_kernel<<<nb, kShThreads, 0, s>>>(theta, K, make_consts(K), dirs, n, base, dpts, dnrm,
                                               h->partials);
  WGEO_LAUNCH_CHECK();
  sh_finalize_kernel<<<1, 128, 0, s>>>(h->partials, nb, K, dtheta);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

int sh_valid_K(int K) {
  const int l = (int)lround(sqrt((double)K)) - 1;
  return (K >= 1 && (l + 1) * (l + 1) == K && l <= kLmax) ? 1 : 0;
}

}  // namespace wgeo

// ------------------------------------------------ allocation-free adjoint
//
// The same two kernels as launch_sh_backward, with the per-block partial sums
// in a fixed device array of this file instead of a handle's workspace.  The
// array holds kShBlocks x kK doubles (256 x 81 x 8 B = 162 KB): the grid is
// capped at kShBlocks blocks and K at kK = 81 (lmax 8), so every accepted
// call fits.  No slot needs to start at zero: the block kernel writes every
// slot [b * K + k] (b < blocks, k < K) that the final kernel reads.  One array
// per device, shared by all calls on that device: calls that overlap in time
// (different streams, or host threads, without ordering) race on it.

namespace wgeo {

static __device__ __align__(256) double sh_noalloc_scratch[kShBlocks * kK];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // id of the context the address belongs to

// Driver entry points for the id of the current context, looked up once
// through the runtime (no link-time dependency on the driver library).
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

// Unique id of the calling thread's current context (the device's primary
// context once the runtime has been used on it); 0 if it cannot be read.
// Called with g_scratch_mu held.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device.  The first call
// per device (and the first after the device's context was replaced, e.g. by
// cudaDeviceReset) checks that the device is sm_103 and resolves the address
// with cudaGetSymbolAddress, which may also load the module on that device;
// later calls in the same context read the cached pointer.
int noalloc_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return WGEO_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return WGEO_ERR_INVALID_ARG;
  // 0 before the runtime has made a context current on this thread: then the
  // address is resolved (which makes the primary context current) and the id
  // read again afterwards
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    g_scratch_ptr[dev] = nullptr;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
      cudaGetLastError();
      return WGEO_ERR_CUDA;
    }
    if (major * 10 + minor != 103) return WGEO_ERR_NOT_BUILT_FOR_DEVICE;
    void* p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, sh_noalloc_scratch);
    if (rc != cudaSuccess || !p) {
      cudaGetLastError();
      return WGEO_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_scratch_ctx[dev] = ctx ? ctx : current_context_id();
  }
  *out = g_scratch_ptr[dev];
  return WGEO_OK;
}

}  // namespace
}  // namespace wgeo

extern "C" int wgeo_sh_surface_backward_noalloc(const float* theta, int32_t K, const float* dirs, int64_t n,
                                                float base, const float* d_points, const float* d_normals,
                                                float* d_theta, void* stream) {
  using namespace wgeo;
  if (K < 1 || K > kK) return WGEO_ERR_INVALID_ARG;   // the scratch holds at most kK coefficients
  if (!sh_valid_K(K) || n < 0 || !theta || !d_theta || (n > 0 && (!dirs || !d_points || !d_normals)))
    return WGEO_ERR_INVALID_ARG;
  double* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc != WGEO_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    WGEO_CUDA_TRY(cudaMemsetAsync(d_theta, 0, sizeof(float) * K, s));
    return WGEO_OK;
  }
  const int nb = grid_blocks(n, kShThreads, kShBlocks);   // nb * K <= kShBlocks * kK
  sh_backward_kernel<<<nb, kShThreads, 0, s>>>(theta, K, make_consts(K), dirs, n, base, d_points, d_normals,
                                               scratch);
  WGEO_LAUNCH_CHECK();
  sh_finalize_kernel<<<1, 128, 0, s>>>(scratch, nb, K, d_theta);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}
