// Queries of the grid SDF and the adjoint chain (Sec. 2.5, Eqs. 35-39).
//
// Query: trilinear phi and the normalised trilinear stencil normal at q, with
// q clamped into the node hull [lo + h/2, lo + (res - 1/2) h] per axis.
//
// Backward, for the discrete choices of the last forward:
//   1. dphi: grid seed + scatter of the query adjoints; normal seeds pass
//      through n = g / |g| (dg = (I - n n^T) dn / |g|) and the transpose of
//      the gradient stencil.
//   2. distance: phi_o = s_o |p_o - y_o| with y_o = sum_v beta_v P_v on the
//      closest triangle -> dP_v = -s_o dphi_o beta_v (p_o - y_o)/|p_o - y_o|;
//      marching cubes: P = node + eta h e_axis, eta = (c - chi1)/(chi2 - chi1)
//      -> d chi1, d chi2 and dc, fused in the same pass.
//   3. iso-value: c = mean_i chi_hat(x_i) -> dchi at the 8 corners, dx_i.
//   4. adjoint solve L lambda = dchi (L symmetric, Eq. 38), FP64-refined.
//   5. divergence transpose dV = D^T lambda and the splat adjoint per point:
//      dn_i = sum_o alpha_oi dV_o, dx_i += sum_o (n_i . dV_o) d alpha_oi / dx_i.
// Scatters use FP64 atomics into FP64 grids.
#include <algorithm>

#include "wgeo_internal.cuh"

namespace wgeo {

namespace {

struct QParams {
  double lo[3];
  double h;
  int res;
  float lo_hi[3], lo_lo[3];   // lo and 1 / h as float-float pairs (trilinear cells off the FP64 pipe)
  float ih_hi, ih_lo;
};

__device__ __forceinline__ int64_t lin3(int i, int j, int k, int n) {
  return ((int64_t)k * n + j) * n + i;
}

// Trilinear cell and weights of a query; dw[c][a] = d w_c / d q_a (0 on clamped axes).
// The node coordinate is float-float (node_coord_ff): no FP64 arithmetic,
// which this GPU runs at a small fraction of its FP32 rate.
__device__ __forceinline__ void trilinear(const float* q, const QParams& g, int i0[3], float w[8],
                                          float dw[8][3]) {
  float t[3], dt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 u = node_coord_ff(q[a], g.lo_hi[a], g.lo_lo[a], g.ih_hi, g.ih_lo);
    const bool cl = node_cell_ff(u, g.res, i0[a], t[a]);
    dt[a] = cl ? 0.f : g.ih_hi;
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
    const float fx = bx ? t[0] : 1.f - t[0], fy = by ? t[1] : 1.f - t[1], fz = bz ? t[2] : 1.f - t[2];
    const float gx = bx ? dt[0] : -dt[0], gy = by ? dt[1] : -dt[1], gz = bz ? dt[2] : -dt[2];
    w[c] = fx * fy * fz;
    dw[c][0] = gx * fy * fz;
    dw[c][1] = fx * gy * fz;
    dw[c][2] = fx * fy * gz;
  }
}

// Stencil gradient of phi at node (i,j,k) (central inside, one-sided 2nd order at the ends).
__device__ __forceinline__ void node_grad(const float* __restrict__ phi, int i, int j, int k, int n,
                                          float inv2h, float g[3]) {
  const int idx[3] = {i, j, k};
  const int64_t t = lin3(i, j, k, n);
  const int64_t st[3] = {1, n, (int64_t)n * n};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float d;
    if (idx[a] == 0)
      d = -3.f * phi[t] + 4.f * phi[t + st[a]] - phi[t + 2 * st[a]];
    else if (idx[a] == n - 1)
      d = 3.f * phi[t] - 4.f * phi[t - st[a]] + phi[t - 2 * st[a]];
    else
      d = phi[t + st[a]] - phi[t - st[a]];
    g[a] = d * inv2h;
  }
}

// Scatter dL/dg at node (i,j,k) through the transpose of the gradient stencil.
__device__ __forceinline__ void scatter_grad_adjoint(float* __restrict__ dphi, int i, int j, int k,
                                                     int n, float inv2h, const float dg[3]) {
  const int idx[3] = {i, j, k};
  const int64_t t = lin3(i, j, k, n);
  const int64_t st[3] = {1, n, (int64_t)n * n};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float v = dg[a] * inv2h;
    if (v == 0.f) continue;
    if (idx[a] == 0) {
      atomicAdd(&dphi[t], -3.f * v);
      atomicAdd(&dphi[t + st[a]], 4.f * v);
      atomicAdd(&dphi[t + 2 * st[a]], -v);
    } else if (idx[a] == n - 1) {
      atomicAdd(&dphi[t], 3.f * v);
      atomicAdd(&dphi[t - st[a]], -4.f * v);
      atomicAdd(&dphi[t - 2 * st[a]], v);
    } else {
      atomicAdd(&dphi[t + st[a]], v);
      atomicAdd(&dphi[t - st[a]], -v);
    }
  }
}

__global__ void query_kernel(const float* __restrict__ q, int64_t m, QParams g,
                             const float* __restrict__ phi, float* __restrict__ sdf_q,
                             float* __restrict__ nrm_q) {
  const int n = g.res;
  const float inv2h = (float)(0.5 / g.h);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float qq[3] = {q[3 * i], q[3 * i + 1], q[3 * i + 2]};
    int i0[3];
    float w[8], dw[8][3];
    trilinear(qq, g, i0, w, dw);
    float s = 0.f;
    float mv[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int x = i0[0] + (c & 1), y = i0[1] + ((c >> 1) & 1), z = i0[2] + (c >> 2);
      s += w[c] * phi[lin3(x, y, z, n)];
      if (nrm_q) {
        float gr[3];
        node_grad(phi, x, y, z, n, inv2h, gr);
        const float m2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
        const float inv = (isfinite(m2) && m2 > 0.f) ? rsqrtf(m2) : 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) mv[a] += w[c] * gr[a] * inv;
      }
    }
    sdf_q[i] = s;
    if (nrm_q) {
      const float m2 = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
      const float inv = (m2 > 0.f) ? rsqrtf(m2) : 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) nrm_q[3 * i + a] = mv[a] * inv;
    }
  }
}

// DN: the loss has a normal term (dnq != null).  Without it the kernel is the
// trilinear part alone, at a fraction of the registers of the normal
// adjoint's corner arrays.
template <bool DN>
__global__ void query_adjoint_kernel(const float* __restrict__ q, int64_t m, QParams g,
                                     const float* __restrict__ phi, const float* __restrict__ dsq,
                                     const float* __restrict__ dnq, float* __restrict__ dphi,
                                     float* __restrict__ dq) {
  const int n = g.res;
  const float inv2h = (float)(0.5 / g.h);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float qq[3] = {q[3 * i], q[3 * i + 1], q[3 * i + 2]};
    int i0[3];
    float w[8], dw[8][3];
    trilinear(qq, g, i0, w, dw);
    float dqa[3] = {0.f, 0.f, 0.f};
    if (dsq) {
      const float gs = dsq[i];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t o = lin3(i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + (c >> 2), n);
        if (gs != 0.f) atomicAdd(&dphi[o], w[c] * gs);
        const float pv = phi[o];
#pragma unroll
        for (int a = 0; a < 3; ++a) dqa[a] += dw[c][a] * pv * gs;
      }
    }
    if (DN && dnq) {
      // recompute the corner normals and the interpolated m
      float nc[8][3], gm[8];
      float mv[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float gr[3];
        node_grad(phi, i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + (c >> 2), n, inv2h, gr);
        const float m2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
        const bool ok = isfinite(m2) && m2 > 0.f;
        gm[c] = ok ? sqrtf(m2) : 0.f;
        const float inv = ok ? 1.f / gm[c] : 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          nc[c][a] = gr[a] * inv;
          mv[a] += w[c] * nc[c][a];
        }
      }
      const float mm = sqrtf(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
      if (mm > 0.f) {
        const float nq[3] = {mv[0] / mm, mv[1] / mm, mv[2] / mm};
        const float gq[3] = {dnq[3 * i], dnq[3 * i + 1], dnq[3 * i + 2]};
        const float pr = nq[0] * gq[0] + nq[1] * gq[1] + nq[2] * gq[2];
        const float dm[3] = {(gq[0] - nq[0] * pr) / mm, (gq[1] - nq[1] * pr) / mm,
                             (gq[2] - nq[2] * pr) / mm};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float nd = nc[c][0] * dm[0] + nc[c][1] * dm[1] + nc[c][2] * dm[2];
#pragma unroll
          for (int a = 0; a < 3; ++a) dqa[a] += dw[c][a] * nd;
          if (gm[c] > 0.f) {
            // dn_c = w_c dm ; dg_c = (I - n n^T) dn_c / |g_c|
            const float wd[3] = {w[c] * dm[0], w[c] * dm[1], w[c] * dm[2]};
            const float pn = nc[c][0] * wd[0] + nc[c][1] * wd[1] + nc[c][2] * wd[2];
            const float dg[3] = {(wd[0] - nc[c][0] * pn) / gm[c], (wd[1] - nc[c][1] * pn) / gm[c],
                                 (wd[2] - nc[c][2] * pn) / gm[c]};
            scatter_grad_adjoint(dphi, i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + (c >> 2), n, inv2h,
                                 dg);
          }
        }
      }
    }
    if (dq) {
#pragma unroll
      for (int a = 0; a < 3; ++a) dq[3 * i + a] = dqa[a];
    }
  }
}

__global__ void grid_seed_kernel(const float* __restrict__ dsg, const float* __restrict__ dng,
                                 const float* __restrict__ phi, QParams g, float* __restrict__ dphi) {
  const int n = g.res;
  const int64_t N = (int64_t)n * n * n;
  const float inv2h = (float)(0.5 / g.h);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (dsg) {
      const float v = dsg[t];
      if (v != 0.f) atomicAdd(&dphi[t], v);
    }
    if (dng) {
      const float dn[3] = {dng[t], dng[N + t], dng[2 * N + t]};
      if (dn[0] == 0.f && dn[1] == 0.f && dn[2] == 0.f) continue;
      const int i = (int)(t % n), j = (int)((t / n) % n), k = (int)(t / ((int64_t)n * n));
      float gr[3];
      node_grad(phi, i, j, k, n, inv2h, gr);
      const float m2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
      if (!(isfinite(m2) && m2 > 0.f)) continue;
      const float gm = sqrtf(m2);
      const float nv[3] = {gr[0] / gm, gr[1] / gm, gr[2] / gm};
      const float pn = nv[0] * dn[0] + nv[1] * dn[1] + nv[2] * dn[2];
      const float dg[3] = {(dn[0] - nv[0] * pn) / gm, (dn[1] - nv[1] * pn) / gm, (dn[2] - nv[2] * pn) / gm};
      scatter_grad_adjoint(dphi, i, j, k, n, inv2h, dg);
    }
  }
}

// Distance + marching-cubes adjoint, one thread per node with a nonzero dphi.
// FP32 arithmetic per node; FP64 only in the scatter (atomics) and the dc sum.
// Per node with dL/dphi != 0: phi = s |p - y| with y the closest point of the
// node's triangle (Eqs. 33-34), y = sum_v beta_v P_v, and each vertex P_v on
// the cube edge (chi1, chi2) at eta = (c - chi1) / (chi2 - chi1) (Eq. 28):
// dL/dP_v = -s dphi beta_v u (u the unit vector from y to p), scattered to
// dL/dchi1, dL/dchi2 and dL/dc.  The closest point comes from the triangle's
// search record, as in the forward search; node coordinates from per-axis
// tables (the forward's float positions), the sign test against the
// smallest float not below c, c - chi1 from c as a float-float pair, and the
// dL/dc sum in float-float, so no node needs the FP64 pipe.  When the
// forward kept the vertices' low parts (tris_lo) and solved in float-float
// (chiff), the closest point is taken from p - a with a's low part, on the
// search record whose edge vectors come from the ~48-bit vertices, and the
// indicator values of each vertex's cube edge carry their float-float low
// parts: the weights then follow the refined surface, not its float32
// rounding, which a far node's closest point would amplify by distance over
// edge length.

// LIST = false: every node with a seed; a node whose closest triangle is a
// sliver (its float32 weights would lose their digits) is appended to
// `slivers` instead.  LIST = true: the listed nodes, weights and direction in
// FP64.  Two passes, so the rare FP64 work does not stall whole warps.
template <bool LIST>
__global__ void sdf_mc_adjoint_kernel(const float* __restrict__ dphi, const int* __restrict__ ctri,
                                      const float* __restrict__ chi, ChiFF chiff, const DevState* __restrict__ st,
                                      const Tri* __restrict__ tris, const Tri* __restrict__ tris_lo,
                                      const float4* __restrict__ tris_s, QParams g,
                                      double* __restrict__ dchi, double* __restrict__ partials,
                                      int* __restrict__ slivers, unsigned* __restrict__ nsliver) {
  __shared__ double red[32];
  __shared__ float s_ax[3][kMaxRes];
  const int n = g.res;
  for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
    const int a = t / n, i = t % n;
    s_ax[a][i] = (float)(g.lo[a] + (i + 0.5) * g.h);
  }
  __syncthreads();
  const double cd = st->c;
  const float cf = st->c_up;
  const float c_hi = (float)cd, c_lo = (float)(cd - (double)c_hi);
  const float hf = (float)g.h;
  const unsigned un = (unsigned)n;
  const unsigned N = LIST ? *nsliver : un * un * un;
  const float2* __restrict__ xff = chiff.p[0] ? chiff.p[st->fwd.xidx] : nullptr;
  float2 dcacc = make_float2(0.f, 0.f);   // dL/dc: terms of both signs that nearly cancel
  for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < N; it += gridDim.x * blockDim.x) {
    const unsigned o = LIST ? (unsigned)slivers[it] : it;
    const float gphi = dphi[o];
    if (gphi == 0.f) continue;   // most nodes carry no seed
    const int t = ctri[o];
    if (t < 0) continue;
    const unsigned row = o / un;
    const int i = (int)(o - row * un), j = (int)(row % un), k = (int)(row / un);
    const float3 p = make_float3(s_ax[0][i], s_ax[1][j], s_ax[2][k]);
    const float4* rec = tris_s + kTriRec * (int64_t)t;
    const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
    float u[3], bw[3];
    const Tri tr = tris[t];
    if (!LIST) {
      if (!(r0.w * r2.w * r3.w < kSliverKappa)) {
        slivers[atomicAdd(nsliver, 1u)] = (int)o;
        continue;
      }
      float3 ap = make_float3(p.x - r0.x, p.y - r0.y, p.z - r0.z);
      if (tris_lo) {
        const float4 al = tris_lo[t].a;
        ap = make_float3(ap.x - al.x, ap.y - al.y, ap.z - al.z);
      }
      const float d1 = r1.x * ap.x + r1.y * ap.y + r1.z * ap.z;
      const float d2 = r2.x * ap.x + r2.y * ap.y + r2.z * ap.z;
      float v, w;
      rec_weights(ap, d1, d2, r0, r1, r2, r3, v, w);
      const float rx = ap.x - v * r1.x - w * r2.x;
      const float ry = ap.y - v * r1.y - w * r2.y;
      const float rz = ap.z - v * r1.z - w * r2.z;
      const float dd = rx * rx + ry * ry + rz * rz;
      if (!(dd > 0.f)) continue;
      const float invd = rsqrtf(dd);
      u[0] = rx * invd, u[1] = ry * invd, u[2] = rz * invd;
      bw[0] = fmaxf(1.f - v - w, 0.f), bw[1] = v, bw[2] = w;
    } else {
      double ad[3] = {tr.a.x, tr.a.y, tr.a.z}, bd[3] = {tr.b.x, tr.b.y, tr.b.z}, cdv[3] = {tr.c.x, tr.c.y, tr.c.z};
      if (tris_lo) {
        const Tri tl = tris_lo[t];
        ad[0] += tl.a.x, ad[1] += tl.a.y, ad[2] += tl.a.z;
        bd[0] += tl.b.x, bd[1] += tl.b.y, bd[2] += tl.b.z;
        cdv[0] += tl.c.x, cdv[1] += tl.c.y, cdv[2] += tl.c.z;
      }
      const double pd[3] = {p.x, p.y, p.z};
      double bw64[3], dir64[3];
      if (!(closest_point_fp64(pd, ad, bd, cdv, bw64, dir64) > 0.0)) continue;
      for (int q = 0; q < 3; ++q) {
        bw[q] = (float)bw64[q];
        u[q] = (float)dir64[q];
      }
    }
    const float sgn = (chi[o] >= cf) ? 1.f : -1.f;
    const float gv[3] = {tr.a.w, tr.b.w, tr.c.w};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (bw[q] == 0.f) continue;
      const unsigned gid = (unsigned)__float_as_int(gv[q]);
      const int ax = (int)(gid % 3u);
      const unsigned pl = gid / 3u;
      const unsigned stv = (ax == 0) ? 1u : (ax == 1 ? un : un * un);
      float den, cm;
      if (xff) {
        // the refined values: hi differences exact or within one rounding, lo parts added
        const float2 f1 = xff[pl], f2 = xff[pl + stv];
        den = __fadd_rn(__fsub_rn(f2.x, f1.x), __fsub_rn(f2.y, f1.y));
        cm = __fadd_rn(__fsub_rn(__fsub_rn(c_hi, f1.x), f1.y), c_lo);
      } else {
        const float c1 = chi[pl], c2 = chi[pl + stv];
        den = c2 - c1;                                             // neighbouring values: exact
        cm = __fadd_rn(__fsub_rn(c_hi, c1), c_lo);                 // c - chi1, keeping c's low bits
      }
      const float eta = cm / den;
      // dL/dP_v[ax] = -s dphi beta_v u[ax];  dP/deta = h e_ax
      const float deta = -sgn * gphi * bw[q] * u[ax] * hf;
      const float wq = deta / den;
      atomicAdd(&dchi[pl], (double)(wq * (eta - 1.f)));
      atomicAdd(&dchi[pl + stv], (double)(-wq * eta));
      dcacc = ff_add_f(dcacc, wq);
    }
  }
  const double s = block_sum<256>((double)dcacc.x + (double)dcacc.y, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void dc_finalize_kernel(const double* __restrict__ partials, int nblocks, DevState* st) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partials[i];
  s = block_sum<1024>(s, red);
  if (threadIdx.x == 0) st->dc = s;
}

// Adds a chunk's block partials of dL/dc to the running sum (chunks in order).
__global__ void dc_add_kernel(const double* __restrict__ partials, int nblocks, DevState* st) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partials[i];
  s = block_sum<1024>(s, red);
  if (threadIdx.x == 0) st->dc += s;
}

// Adjoint of exact off-grid queries: phi(q) = s |q - y|, y = sum_v beta_v P_v
// on the query's closest triangle, so dL/dP_v = -dL/dphi beta_v s u with
// s u = (grad phi)(q), the gradient the forward query wrote; then through
// the marching-cubes vertex P_v = node + eta h e_ax to chi and c, as for the
// node seeds.  d_q = dL/dphi (grad phi)(q).  Queries with a non-finite
// distance or none (empty surface) contribute nothing.
__global__ void exact_adjoint_kernel(const float* __restrict__ q, int nq, const float* __restrict__ g_sdf,
                                     const float* __restrict__ tsdf, const float* __restrict__ tgrad,
                                     const int* __restrict__ ttri, const float* __restrict__ chi, ChiFF chiff,
                                     const DevState* __restrict__ st, const Tri* __restrict__ tris,
                                     const Tri* __restrict__ tris_lo,
                                     const float4* __restrict__ tris_s, QParams g, double* __restrict__ dchi,
                                     double* __restrict__ partials, float* __restrict__ d_q) {
  __shared__ double red[32];
  const double cd = st->c;
  const float c_hi = (float)cd, c_lo = (float)(cd - (double)c_hi);
  const float hf = (float)g.h;
  const unsigned un = (unsigned)g.res;
  const float2* __restrict__ xff = chiff.p[0] ? chiff.p[st->fwd.xidx] : nullptr;
  float2 dcacc = make_float2(0.f, 0.f);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
    const float gi = g_sdf[i], d = tsdf[i];
    const int t = ttri[i];
    const float us[3] = {tgrad[3 * (int64_t)i], tgrad[3 * (int64_t)i + 1], tgrad[3 * (int64_t)i + 2]};
    const bool ok = gi != 0.f && isfinite(d) && t >= 0;
    if (d_q) {
      d_q[3 * (int64_t)i] = ok ? gi * us[0] : 0.f;
      d_q[3 * (int64_t)i + 1] = ok ? gi * us[1] : 0.f;
      d_q[3 * (int64_t)i + 2] = ok ? gi * us[2] : 0.f;
    }
    if (!ok || d == 0.f) continue;
    const float3 p = make_float3(q[3 * (int64_t)i], q[3 * (int64_t)i + 1], q[3 * (int64_t)i + 2]);
    const float4* rec = tris_s + kTriRec * (int64_t)t;
    const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
    float3 ap = make_float3(p.x - r0.x, p.y - r0.y, p.z - r0.z);
    if (tris_lo) {
      const float4 al = tris_lo[t].a;
      ap = make_float3(ap.x - al.x, ap.y - al.y, ap.z - al.z);
    }
    const float d1 = r1.x * ap.x + r1.y * ap.y + r1.z * ap.z;
    const float d2 = r2.x * ap.x + r2.y * ap.y + r2.z * ap.z;
    float v, w;
    rec_weights(ap, d1, d2, r0, r1, r2, r3, v, w);
    float bw[3] = {fmaxf(1.f - v - w, 0.f), v, w};
    const Tri tr = tris[t];
    if (!(r0.w * r2.w * r3.w < kSliverKappa)) {
      double ad[3] = {tr.a.x, tr.a.y, tr.a.z}, bd[3] = {tr.b.x, tr.b.y, tr.b.z}, cdv[3] = {tr.c.x, tr.c.y, tr.c.z};
      if (tris_lo) {
        const Tri tl = tris_lo[t];
        ad[0] += tl.a.x, ad[1] += tl.a.y, ad[2] += tl.a.z;
        bd[0] += tl.b.x, bd[1] += tl.b.y, bd[2] += tl.b.z;
        cdv[0] += tl.c.x, cdv[1] += tl.c.y, cdv[2] += tl.c.z;
      }
      const double pd[3] = {p.x, p.y, p.z};
      double bw64[3], dir64[3];
      closest_point_fp64(pd, ad, bd, cdv, bw64, dir64);
      for (int q = 0; q < 3; ++q) bw[q] = (float)bw64[q];
    }
    const float gv[3] = {tr.a.w, tr.b.w, tr.c.w};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (bw[k] == 0.f) continue;
      const unsigned gid = (unsigned)__float_as_int(gv[k]);
      const int ax = (int)(gid % 3u);
      const unsigned pl = gid / 3u;
      const unsigned stv = (ax == 0) ? 1u : (ax == 1 ? un : un * un);
      float den, cm;
      if (xff) {
        const float2 f1 = xff[pl], f2 = xff[pl + stv];
        den = __fadd_rn(__fsub_rn(f2.x, f1.x), __fsub_rn(f2.y, f1.y));
        cm = __fadd_rn(__fsub_rn(__fsub_rn(c_hi, f1.x), f1.y), c_lo);
      } else {
        const float c1 = chi[pl], c2 = chi[pl + stv];
        den = c2 - c1;
        cm = __fadd_rn(__fsub_rn(c_hi, c1), c_lo);
      }
      const float eta = cm / den;
      const float deta = -gi * bw[k] * us[ax] * hf;
      const float wq = deta / den;
      atomicAdd(&dchi[pl], (double)(wq * (eta - 1.f)));
      atomicAdd(&dchi[pl + stv], (double)(-wq * eta));
      dcacc = ff_add_f(dcacc, wq);
    }
  }
  const double s = block_sum<256>((double)dcacc.x + (double)dcacc.y, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Iso-value adjoint: dchi += dc/N_p * w at the 8 corners; d_points = dc/N_p * sum dw chi.
__global__ void iso_adjoint_kernel(const int* __restrict__ pcell, const float4* __restrict__ pfrac,
                                   int64_t np, const float* __restrict__ chi,
                                   const DevState* __restrict__ st, QParams g,
                                   double* __restrict__ dchi, float* __restrict__ dpts) {
  const int n = g.res;
  const double scale = st->npts > 0 ? st->dc / (double)st->npts : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int pc = pcell[i];
    if (pc < 0 || scale == 0.0) {
      dpts[3 * i] = 0.f;
      dpts[3 * i + 1] = 0.f;
      dpts[3 * i + 2] = 0.f;
      continue;
    }
    const float4 fr = pfrac[i];
    const int b[3] = {cell_x(pc), cell_y(pc), cell_z(pc)};
    const float f[3] = {fr.x, fr.y, fr.z};
    int i0[3];
    double t[3], dt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double u = (double)b[a] + (double)f[a] - 0.5;
      const bool cl = (u < 0.0) || (u > (double)(n - 1));
      u = fmin(fmax(u, 0.0), (double)(n - 1));
      int fl = (int)floor(u);
      fl = min(fl, n - 2);
      i0[a] = fl;
      t[a] = u - fl;
      dt[a] = cl ? 0.0 : 1.0 / g.h;
    }
    double dx[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
      const double fx = bx ? t[0] : 1 - t[0], fy = by ? t[1] : 1 - t[1], fz = bz ? t[2] : 1 - t[2];
      const double gx = bx ? dt[0] : -dt[0], gy = by ? dt[1] : -dt[1], gz = bz ? dt[2] : -dt[2];
      const int64_t o = lin3(i0[0] + bx, i0[1] + by, i0[2] + bz, n);
      atomicAdd(&dchi[o], scale * fx * fy * fz);
      const double cv = (double)chi[o];
      dx[0] += gx * fy * fz * cv;
      dx[1] += fx * gy * fz * cv;
      dx[2] += fx * fy * gz * cv;
    }
    dpts[3 * i] = (float)(scale * dx[0]);
    dpts[3 * i + 1] = (float)(scale * dx[1]);
    dpts[3 * i + 2] = (float)(scale * dx[2]);
  }
}

// dV_o = D^T lambda at cell (x,y,z): 1/2 (lambda_o - lambda_{o+e}) on interior
// faces o+1/2 plus 1/2 (lambda_{o-e} - lambda_o) on interior faces o-1/2;
// lambda is float-float, the differences are formed exactly.
__device__ __forceinline__ void dV_at(const float2* __restrict__ lam, int x, int y, int z, int n,
                                      float dv[3]) {
  const int idx[3] = {x, y, z};
  const int64_t o = lin3(x, y, z, n);
  const int64_t st[3] = {1, n, (int64_t)n * n};
  const float2 lo = lam[o];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float v = 0.f;
    if (idx[a] + 1 < n) {
      const float2 d = ff_sub(lo, lam[o + st[a]]);
      v += 0.5f * (d.x + d.y);
    }
    if (idx[a] - 1 >= 0) {
      const float2 d = ff_sub(lam[o - st[a]], lo);
      v += 0.5f * (d.x + d.y);
    }
    dv[a] = v;
  }
}

// The unlumped Galerkin right-hand side b = sum_xi M M D_xi V_xi has the
// adjoint dV_xi = M M D_xi^T lambda (M symmetric, the walls mirrored): the
// D^T lambda of the 9 transverse neighbours, weighted {1, 4, 1} / 6 per axis.
__device__ __forceinline__ int q1_mass_w(int d, int c, int n) {
  if (d < 0) return c > 0 ? 1 : 0;
  if (d > 0) return c < n - 1 ? 1 : 0;
  return 4 + (c == 0 ? 1 : 0) + (c == n - 1 ? 1 : 0);
}

__device__ __forceinline__ void dV_q1_at(const float2* __restrict__ lam, int x, int y, int z, int n, float dv[3]) {
  const int idx[3] = {x, y, z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ab = a == 0 ? 1 : 0, ac = a == 2 ? 1 : 2;
    float v = 0.f;
    for (int db = -1; db <= 1; ++db) {
      const int wb = q1_mass_w(db, idx[ab], n);
      if (!wb) continue;
      for (int dc = -1; dc <= 1; ++dc) {
        const int wc = q1_mass_w(dc, idx[ac], n);
        if (!wc) continue;
        int q[3] = {x, y, z};
        q[ab] += db;
        q[ac] += dc;
        float d[3];
        dV_at(lam, q[0], q[1], q[2], n, d);
        v += (float)(wb * wc) * d[a];
      }
    }
    dv[a] = v * (1.f / 36.f);
  }
}

template <bool Q1>
__global__ void splat_adjoint_kernel(const int* __restrict__ pcell, const float4* __restrict__ pfrac,
                                     const float4* __restrict__ pnrm, int64_t np,
                                     const float2* __restrict__ lam0, const float2* __restrict__ lam1,
                                     const int* __restrict__ lam_idx, QParams g,
                                     float* __restrict__ dpts, float* __restrict__ dnrm) {
  const float2* __restrict__ lam = (*lam_idx) ? lam1 : lam0;
  const int n = g.res;
  const float inv2h = (float)(0.5 / g.h);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int pc = pcell[i];
    if (pc < 0) {
      dnrm[3 * i] = 0.f;
      dnrm[3 * i + 1] = 0.f;
      dnrm[3 * i + 2] = 0.f;
      continue;
    }
    const float4 fr = pfrac[i];
    const float4 nv = pnrm[i];
    const int b[3] = {cell_x(pc), cell_y(pc), cell_z(pc)};
    const float f[3] = {fr.x, fr.y, fr.z};
    const float nn[3] = {nv.x, nv.y, nv.z};
    float fac[3][3], dfac[3][3];
    bool ing[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float s = f[a] - 0.5f - (float)(d - 1);   // (x - c_o) / h
        const float arg = 1.f - 0.5f * fabsf(s);
        fac[a][d] = 0.5f * fmaxf(0.f, arg);
        dfac[a][d] = (arg > 0.f) ? -0.5f * (float)((s > 0.f) - (s < 0.f)) * inv2h : 0.f;
        const int o = b[a] + d - 1;
        ing[a][d] = (o >= 0) && (o < n);
      }
    }
    float S = 0.f, dS[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int dx = q % 3, dy = (q / 3) % 3, dz = q / 9;
      if (!(ing[0][dx] && ing[1][dy] && ing[2][dz])) continue;
      if (q == 13) {
        S += 0.5f;
        continue;
      }
      S += fac[0][dx] * fac[1][dy] * fac[2][dz];
      dS[0] += dfac[0][dx] * fac[1][dy] * fac[2][dz];
      dS[1] += fac[0][dx] * dfac[1][dy] * fac[2][dz];
      dS[2] += fac[0][dx] * fac[1][dy] * dfac[2][dz];
    }
    const float invS = 1.f / S;
    float gdn[3] = {0.f, 0.f, 0.f}, gdx[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int dx = q % 3, dy = (q / 3) % 3, dz = q / 9;
      if (!(ing[0][dx] && ing[1][dy] && ing[2][dz])) continue;
      float dv[3];
      if (Q1)
        dV_q1_at(lam, b[0] + dx - 1, b[1] + dy - 1, b[2] + dz - 1, n, dv);
      else
        dV_at(lam, b[0] + dx - 1, b[1] + dy - 1, b[2] + dz - 1, n, dv);
      float a, da[3];
      if (q == 13) {
        a = 0.5f;
        da[0] = da[1] = da[2] = 0.f;
      } else {
        a = fac[0][dx] * fac[1][dy] * fac[2][dz];
        da[0] = dfac[0][dx] * fac[1][dy] * fac[2][dz];
        da[1] = fac[0][dx] * dfac[1][dy] * fac[2][dz];
        da[2] = fac[0][dx] * fac[1][dy] * dfac[2][dz];
      }
      const float alpha = a * invS;
      const float wdot = nn[0] * dv[0] + nn[1] * dv[1] + nn[2] * dv[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gdn[c] += alpha * dv[c];
        gdx[c] += wdot * (da[c] - alpha * dS[c]) * invS;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dnrm[3 * i + c] = gdn[c];
      dpts[3 * i + c] = dpts[3 * i + c] + gdx[c];
    }
  }
}


QParams qparams(const wgeo_handle* h) {
  QParams g;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = h->lo[a];
    g.lo_hi[a] = (float)h->lo[a];
    g.lo_lo[a] = (float)(h->lo[a] - (double)g.lo_hi[a]);
  }
  g.h = h->h;
  g.res = h->res;
  const double ih = 1.0 / h->h;
  g.ih_hi = (float)ih;
  g.ih_lo = (float)(ih - (double)g.ih_hi);
  return g;
}

}  // namespace

int launch_query(wgeo_handle* h, const float* q, int64_t m, float* sdf_q, float* nrm_q, cudaStream_t s) {
  if (m == 0) return WGEO_OK;
  query_kernel<<<grid_blocks(m, 256, 152 * 32), 256, 0, s>>>(q, m, qparams(h), h->phi, sdf_q, nrm_q);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

namespace {

// Seeds on the grid (phi and normal seeds): dphi cleared and filled.
int backward_grid_seeds(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, cudaStream_t s) {
  const int64_t N = (int64_t)h->res * h->res * h->res;
  WGEO_CUDA_TRY(cudaMemsetAsync(h->dphi, 0, sizeof(float) * N, s));
  WGEO_CUDA_TRY(cudaMemsetAsync(h->dchi64, 0, sizeof(double) * N, s));
  if (d_sdf_grid || d_nrm_grid) {
    grid_seed_kernel<<<grid_blocks(N, 256, 152 * 32), 256, 0, s>>>(d_sdf_grid, d_nrm_grid, h->phi, qparams(h),
                                                                   h->dphi);
    WGEO_LAUNCH_CHECK();
  }
  return WGEO_OK;
}

// Node phi seeds through the closest triangles and marching cubes to dchi64
// and dL/dc (dstate->dc).
int backward_mesh_nodes(wgeo_handle* h, cudaStream_t s) {
  const int64_t N = (int64_t)h->res * h->res * h->res;
  const int nb = grid_blocks(N, 256, kPartials);
  const int nb2 = 152 * 4;
  // the solver's correction buffer is idle until the adjoint solve: it holds
  // the sliver nodes between the two passes
  int* slivers = reinterpret_cast<int*>(h->e32);
  WGEO_CUDA_TRY(cudaMemsetAsync(&h->dstate->nsliver, 0, sizeof(unsigned), s));
  const ChiFF cff = chiff_of(h);
  sdf_mc_adjoint_kernel<false><<<nb, 256, 0, s>>>(h->dphi, h->ctri, h->chi32, cff, h->dstate, h->tris,
                                                  h->tris_lo, h->tris_s, qparams(h), h->dchi64, h->partials,
                                                  slivers, &h->dstate->nsliver);
  WGEO_LAUNCH_CHECK();
  sdf_mc_adjoint_kernel<true><<<nb2, 256, 0, s>>>(h->dphi, h->ctri, h->chi32, cff, h->dstate, h->tris,
                                                  h->tris_lo, h->tris_s, qparams(h), h->dchi64, h->partials + nb,
                                                  slivers, &h->dstate->nsliver);
  WGEO_LAUNCH_CHECK();
  dc_finalize_kernel<<<1, 1024, 0, s>>>(h->partials, nb + nb2, h->dstate);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

// From dchi64 and dL/dc: iso-value adjoint, adjoint solve, splat adjoint.
int backward_tail(wgeo_handle* h, float* d_points, float* d_normals, cudaStream_t s) {
  const QParams g = qparams(h);
  if (h->npts > 0) {
    iso_adjoint_kernel<<<grid_blocks(h->npts, 256, 152 * 32), 256, 0, s>>>(
        h->pcell, h->pfrac, h->npts, h->chi32, h->dstate, g, h->dchi64, d_points);
    WGEO_LAUNCH_CHECK();
  }
  stage_end(h, kStBwdSurf, h->bwd_slot, s);
  int slot = stage_begin(h, kStBwdSolve, s);
  int rc = launch_solve(h, h->res, 1, true, s);
  if (rc) return rc;
  stage_end(h, kStBwdSolve, slot, s);
  slot = stage_begin(h, kStBwdSplat, s);
  if (h->npts > 0) {
    if (h->opt.galerkin)
      splat_adjoint_kernel<true><<<grid_blocks(h->npts, 128, 152 * 64), 128, 0, s>>>(
          h->pcell, h->pfrac, h->pnrm, h->npts, h->lamff[0], h->lamff[1], &h->dstate->bwd.xidx, g,
          d_points, d_normals);
    else
      splat_adjoint_kernel<false><<<grid_blocks(h->npts, 128, 152 * 64), 128, 0, s>>>(
          h->pcell, h->pfrac, h->pnrm, h->npts, h->lamff[0], h->lamff[1], &h->dstate->bwd.xidx, g,
          d_points, d_normals);
    WGEO_LAUNCH_CHECK();
  }
  stage_end(h, kStBwdSplat, slot, s);
  return WGEO_OK;
}

}  // namespace

int launch_backward(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                    const float* d_sdf_q, const float* d_nrm_q, int64_t m, float* d_points,
                    float* d_normals, float* d_q, cudaStream_t s) {
  int slot = stage_begin(h, kStBwdSeed, s);
  int rc = backward_grid_seeds(h, d_sdf_grid, d_nrm_grid, s);
  if (rc) return rc;
  if (m > 0 && q && (d_sdf_q || d_nrm_q || d_q)) {
    if (d_nrm_q)
      query_adjoint_kernel<true><<<grid_blocks(m, 256, 152 * 32), 256, 0, s>>>(q, m, qparams(h), h->phi, d_sdf_q,
                                                                               d_nrm_q, h->dphi, d_q);
    else
      query_adjoint_kernel<false><<<grid_blocks(m, 256, 152 * 32), 256, 0, s>>>(q, m, qparams(h), h->phi, d_sdf_q,
                                                                                nullptr, h->dphi, d_q);
    WGEO_LAUNCH_CHECK();
  }
  stage_end(h, kStBwdSeed, slot, s);
  h->bwd_slot = stage_begin(h, kStBwdSurf, s);
  rc = backward_mesh_nodes(h, s);
  if (rc) return rc;
  return backward_tail(h, d_points, d_normals, s);
}

int launch_backward_exact(wgeo_handle* h, const float* d_sdf_grid, const float* d_nrm_grid, const float* q,
                          const float* d_sdf_q, int64_t m, float* d_points, float* d_normals, float* d_q,
                          cudaStream_t s) {
  int slot = stage_begin(h, kStBwdSeed, s);
  int rc = backward_grid_seeds(h, d_sdf_grid, d_nrm_grid, s);
  if (rc) return rc;
  stage_end(h, kStBwdSeed, slot, s);
  h->bwd_slot = stage_begin(h, kStBwdSurf, s);
  rc = backward_mesh_nodes(h, s);
  if (rc) return rc;
  // exact queries, chunk by chunk: the forward query again (distance, the
  // gradient and the closest triangle, held in the point-grid scratch that
  // the query's sort no longer needs), then their adjoint
  const int64_t P = h->dp_points;
  float* tsdf = reinterpret_cast<float*>(h->dp_tmp);
  float* tgrad = tsdf + P;
  int* ttri = h->dp_key;
  for (int64_t c0 = 0; c0 < m && d_sdf_q; c0 += P) {
    const int nq = (int)std::min<int64_t>(P, m - c0);
    rc = launch_query_exact_chunk(h, q + 3 * c0, nq, tsdf, tgrad, ttri, s);
    if (rc) return rc;
    const int nb = grid_blocks(nq, 256, kPartials);
    exact_adjoint_kernel<<<nb, 256, 0, s>>>(q + 3 * c0, nq, d_sdf_q + c0, tsdf, tgrad, ttri, h->chi32,
                                            chiff_of(h), h->dstate, h->tris, h->tris_lo, h->tris_s, qparams(h),
                                            h->dchi64, h->partials, d_q ? d_q + 3 * c0 : nullptr);
    WGEO_LAUNCH_CHECK();
    dc_add_kernel<<<1, 1024, 0, s>>>(h->partials, nb, h->dstate);
    WGEO_LAUNCH_CHECK();
  }
  if (!d_sdf_q && d_q && m > 0) WGEO_CUDA_TRY(cudaMemsetAsync(d_q, 0, sizeof(float) * 3 * (size_t)m, s));
  return backward_tail(h, d_points, d_normals, s);
}

}  // namespace wgeo

namespace wgeo {

namespace {

__global__ void export_f64_kernel(const double* __restrict__ src, int64_t N, float* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)src[t];
}

__global__ void export_ff_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                 const int* __restrict__ idx, int64_t N, float* __restrict__ out) {
  const float2* __restrict__ src = (*idx) ? b : a;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = src[t].x + src[t].y;
}

}  // namespace

// Backward intermediates as float32: 3 dL/dphi, 4 dL/dchi, 5 lambda.
int launch_export_adjoint(wgeo_handle* h, int which, float* out, cudaStream_t s) {
  const int64_t N = (int64_t)h->res * h->res * h->res;
  const int gb = grid_blocks(N, 256, 152 * 32);
  if (which == 3)
    WGEO_CUDA_TRY(cudaMemcpyAsync(out, h->dphi, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
  else if (which == 4)
    export_f64_kernel<<<gb, 256, 0, s>>>(h->dchi64, N, out);
  else
    export_ff_kernel<<<gb, 256, 0, s>>>(h->lamff[0], h->lamff[1], &h->dstate->bwd.xidx, N, out);
  WGEO_LAUNCH_CHECK();
  return WGEO_OK;
}

}  // namespace wgeo
