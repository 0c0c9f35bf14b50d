// Exclusive prefix sum of int32 counts (tile and brick offsets).
// Hierarchical: 1024-element blocks scanned with warp shuffles, block totals
// scanned recursively, then added back.  out has n + 1 entries; out[n] = total.
#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

constexpr int kScanThreads = 1024;

__global__ void scan_block_kernel(const int* __restrict__ in, int* __restrict__ out, int n,
                                  int* __restrict__ block_sums) {
  __shared__ int warp_tot[32];
  const int i = blockIdx.x * kScanThreads + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int v = (i < n) ? in[i] : 0;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int t = warp_tot[lane];
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) block_sums[blockIdx.x] = ti;
  }
  __syncthreads();
  if (i < n) out[i] = incl - v + warp_tot[w];
}

__global__ void add_offsets_kernel(int* __restrict__ out, int n, const int* __restrict__ offs) {
  const int i = blockIdx.x * kScanThreads + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

__global__ void write_total_kernel(const int* __restrict__ in, int* __restrict__ out, int n) {
  out[n] = (n > 0) ? out[n - 1] + in[n - 1] : 0;
}

}  // namespace

size_t scan_tmp_size(int n) {
  size_t total = 0;
  int m = n;
  while (m > 1) {
    int nb = div_up(m, kScanThreads);
    total += (size_t)nb * 2 + 2;
    m = nb;
  }
  return total + 4;
}

static int scan_rec(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
  if (n <= 0) return WGEO_OK;
  const int nb = div_up(n, kScanThreads);
  int* sums = tmp;
  int* sums_scanned = tmp + nb;
  scan_block_kernel<<<nb, kScanThreads, 0, s>>>(in, out, n, sums);
  WGEO_LAUNCH_CHECK();
  if (nb > 1) {
    int rc = scan_rec(sums, sums_scanned, nb, tmp + 2 * nb + 2, s);
    if (rc) return rc;
    add_offsets_kernel<<<nb, kScanThreads, 0, s>>>(out, n, sums_scanned);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

int exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
  int rc = scan_rec(in, out, n, tmp, s);
  if (rc) return rc;
  write_total_kernel<<<1, 1, 0, s>>>(in, out, n);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

}  // namespace wgeo
