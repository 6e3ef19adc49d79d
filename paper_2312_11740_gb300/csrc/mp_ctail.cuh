// Coarse tail of the FP32 V-cycle on a thread-block cluster (A6-A9).
//
// Below a few hundred thousand cells every V-cycle kernel is latency-bound:
// a level of 32^3 cells costs a launch of ~5 us per red-black sweep whatever
// its size.  The one-CTA tail (k_tail) removes the launches for the levels
// that fit one CTA's shared memory (<= 16^3).  This kernel takes one level
// more: a cluster of CT_CTAS CTAs keeps the top level (32^3 at 256^3) and
// every coarser level in distributed shared memory, split in z-slabs, and runs
// the sweeps, restrictions, prolongations and the coarsest solve with cluster
// barriers in place of launches.  A cell's z-neighbours in another CTA's slab
// are read through distributed shared memory.
//
// Same algorithm and arithmetic per cell as k_tail: red-black Gauss-Seidel
// on FP32 faces with the stored FP32 1/diag, colour c0 = 0 first on the way
// down and last on the way up (a symmetric preconditioner), difference-form
// residuals, restriction by half the sum of the 8 children, piecewise-
// constant prolongation, and the dense FP64 coarsest inverse.
//
// Slabs: level l has ppc = max(1, nz / CT_CTAS) planes per CTA; CTA r owns
// planes [r ppc, (r + 1) ppc) that exist (with nz < CT_CTAS, CTA r owns plane
// r if r < nz).  Every CTA lays out its slab arrays at the same offsets, so a
// plane's owner and offset follow from its index alone.  Requirements
// (checked by the host): every level's nz a multiple of CT_CTAS or at most
// CT_CTAS; the slabs fit shared memory; the coarsest level has <= 512 cells.
#pragma once

#include <cooperative_groups.h>

namespace mp {

namespace cgx = cooperative_groups;

constexpr int CT_CTAS = 8, CTL_THREADS = 1024, CT_MAX_LEVELS = 8, CT_MAX_COARSE = 512;

struct CtLevel {
  Dims d;
  int n, nu1, nu2;
  int ppc;  // z-planes per CTA
  int off;  // float offset of the level's slab arrays in every CTA's shared memory
  const float *bx, *by, *bz, *idiag, *dd;  // FP32 level arrays (dd null without outflow)
};
struct CtArgs {
  int nlev;  // levels in the cluster tail (the last one is the coarsest)
  CtLevel lv[CT_MAX_LEVELS];
  const double *Minv;
  int singular;  // mean-project the coarsest right-hand side
};

// Floats of one level's slab arrays in one CTA: x, b, wx, wy, 1/diag (ppc
// planes each), wz (ppc + 1 planes: the slab's low z faces and those of the
// plane above it, so a cell's high z face is always local), dd (ppc planes,
// outflow only).
__host__ __device__ inline int ct_slab_floats(const Dims &d, int ppc, bool dd) {
  const int pl = d.nx * d.ny, s = pl * ppc;
  return 5 * s + s + pl + (dd ? s : 0);
}

// Quotient t / d from m = ct_magic(d) (round-up reciprocal, m d - 2^32 < d:
// the high word of t m is exact whenever t d < 2^32; here t and d stay below
// 2^16).  The indexing here divides by runtime sizes in every
// loop; a hardware-free division is a few instructions instead of ~20.
// (d = 1 gives m = 0, which ct_div reads as "the quotient is t")
__device__ __forceinline__ unsigned ct_magic(unsigned d) { return 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int ct_div(int t, unsigned m) {
  return m ? (int)__umulhi((unsigned)t, m) : t;
}

struct CtView {
  float *x, *b, *wx, *wy, *id, *wz, *dd;
  int nx, ny, nz, pl, ppc;
  int k0, own;  // first plane of this CTA's slab, planes it owns (0 at coarse levels)
  unsigned mnx, mny, mhx, mpl, mppc;  // ct_div multipliers of nx, ny, nx / 2, nx ny, ppc
  __device__ CtView(float *base, const CtLevel &l, int rank) {
    nx = l.d.nx, ny = l.d.ny, nz = l.d.nz, pl = nx * ny, ppc = l.ppc;
    const int s = pl * ppc;
    x = base + l.off;
    b = x + s;
    wx = b + s;
    wy = wx + s;
    id = wy + s;
    wz = id + s;
    dd = l.dd ? wz + s + pl : nullptr;
    k0 = rank * ppc;
    own = k0 >= nz ? 0 : min(ppc, nz - k0);
    mnx = ct_magic(nx), mny = ct_magic(ny), mhx = ct_magic(nx > 1 ? nx >> 1 : 1), mpl = ct_magic(pl);
    mppc = ct_magic(ppc);
  }
  __device__ int owner(int k) const { return ct_div(k, mppc); }
  // a plane of array `a` (one of this view's slab arrays) in its owner's slab
  __device__ float *plane(cgx::cluster_group &cl, float *a, int k) const {
    const int r = owner(k);
    return cl.map_shared_rank(a, r) + (size_t)(k - r * ppc) * pl;
  }
};

// One colour of one Gauss-Seidel sweep over this CTA's slab (k_tail's
// half-sweep: the same operand order).  zero: x is taken as zero.
__device__ __forceinline__ void ct_halfsweep(cgx::cluster_group &cl, const CtView &v, int colour,
                                             int zero) {
  if (v.own == 0) return;
  const int nx = v.nx, ny = v.ny, nz = v.nz, pl = v.pl, hx = nx >> 1;
  // x of the planes next to the slab (other CTAs' slabs, or this one's when it
  // holds every plane)
  const int kb = v.k0 == 0 ? nz - 1 : v.k0 - 1, ka = v.k0 + v.own == nz ? 0 : v.k0 + v.own;
  const float *xbelow = v.plane(cl, v.x, kb), *xabove = v.plane(cl, v.x, ka);
  const int half = (v.own * pl) >> 1;
  for (int t = threadIdx.x; t < half; t += CTL_THREADS) {
    const int row = ct_div(t, v.mhx);
    const int kl = ct_div(row, v.mny), j = row - kl * ny, k = v.k0 + kl;
    const int i = 2 * (t - row * hx) + ((j + k + colour) & 1);
    const int c = i + j * nx + kl * pl, cp = i + j * nx;
    const int xp = i == nx - 1 ? c - (nx - 1) : c + 1;
    const int yp = j == ny - 1 ? c - (ny - 1) * nx : c + nx;
    float num = -v.b[c];
    if (!zero) {
      const int xm = i == 0 ? c + (nx - 1) : c - 1;
      const int ym = j == 0 ? c + (ny - 1) * nx : c - nx;
      const float zlo = kl > 0 ? v.x[c - pl] : xbelow[cp];
      const float zhi = kl + 1 < v.own ? v.x[c + pl] : xabove[cp];
      num = fmaf(v.wx[c], v.x[xm], num);
      num = fmaf(v.wx[xp], v.x[xp], num);
      num = fmaf(v.wy[c], v.x[ym], num);
      num = fmaf(v.wy[yp], v.x[yp], num);
      num = fmaf(v.wz[c], zlo, num);
      num = fmaf(v.wz[c + pl], zhi, num);
    }
    v.x[c] = num * v.id[c];
  }
}

// residual b - A x at cell (i, j, k) of a level, any owner (difference form,
// op_at's operand order)
__device__ __forceinline__ float ct_resid(cgx::cluster_group &cl, const CtView &v, int i, int j,
                                          int k) {
  const int nx = v.nx, ny = v.ny, nz = v.nz;
  const int cp = i + j * nx;
  const float *x = v.plane(cl, v.x, k);
  const float *xl = v.plane(cl, v.x, k == 0 ? nz - 1 : k - 1);
  const float *xh = v.plane(cl, v.x, k == nz - 1 ? 0 : k + 1);
  const float *wx = v.plane(cl, v.wx, k), *wy = v.plane(cl, v.wy, k);
  const float *wz = v.plane(cl, v.wz, k);  // + pl: the high faces, in the same slab
  const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const float xc = x[cp];
  float s = wx[cp] * (x[im + j * nx] - xc);
  s = fmaf(wx[ip + j * nx], x[ip + j * nx] - xc, s);
  s = fmaf(wy[cp], x[i + jm * nx] - xc, s);
  s = fmaf(wy[i + jp * nx], x[i + jp * nx] - xc, s);
  s = fmaf(wz[cp], xl[cp] - xc, s);
  s = fmaf(wz[cp + v.pl], xh[cp] - xc, s);
  if (v.dd) s = fmaf(-v.plane(cl, v.dd, k)[cp], xc, s);
  return v.plane(cl, v.b, k)[cp] - s;
}

// x ~= At^-1 rhs on the cluster tail's top level (zero initial guess): one
// symmetric V-cycle over every level the cluster holds.  Launched as one
// cluster of CT_CTAS CTAs; every CTA takes part in every cluster barrier.
// scratch: float offset of CT_MAX_COARSE floats for the gathered coarsest rhs.
__global__ void __launch_bounds__(CTL_THREADS, 1)
k_ctail(CtArgs a, int scratch, const float *__restrict__ rhs, float *__restrict__ xout) {
  griddep_wait();
  cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) float ct_smem[];
  __shared__ double mean_s;
  // this CTA's slabs of the level coefficients, and of the top level's rhs
  for (int l = 0; l < a.nlev; ++l) {
    const CtView v(ct_smem, a.lv[l], rank);
    if (!v.own) continue;
    const CtLevel &g = a.lv[l];
    const size_t g0 = (size_t)v.k0 * v.pl;
    const int s = v.own * v.pl;
    for (int e = threadIdx.x; e < s; e += CTL_THREADS) {
      v.wx[e] = g.bx[g0 + e];
      v.wy[e] = g.by[g0 + e];
      v.wz[e] = g.bz[g0 + e];
      v.id[e] = g.idiag[g0 + e];
      if (v.dd) v.dd[e] = g.dd[g0 + e];
      if (l == 0) v.b[e] = rhs[g0 + e];
    }
    const size_t ga = (size_t)((v.k0 + v.own) % v.nz) * v.pl;  // low faces of the plane above
    for (int e = threadIdx.x; e < v.pl; e += CTL_THREADS) v.wz[s + e] = g.bz[ga + e];
  }
  cl.sync();  // every CTA of the cluster has started and loaded its slabs
  const int last = a.nlev - 1;
  for (int l = 0; l < last; ++l) {  // down
    const CtView v(ct_smem, a.lv[l], rank), vc(ct_smem, a.lv[l + 1], rank);
    for (int s = 0; s < a.lv[l].nu1; ++s) {
      ct_halfsweep(cl, v, 0, s == 0);
      cl.sync();
      ct_halfsweep(cl, v, 1, 0);
      cl.sync();
    }
    for (int e = threadIdx.x; e < vc.own * vc.pl; e += CTL_THREADS) {
      const int kq = ct_div(e, vc.mpl), r = e - kq * vc.pl, J = ct_div(r, vc.mnx);
      const int I = r - J * vc.nx, K = vc.k0 + kq;
      float sum = 0.f;
      for (int q = 0; q < 8; ++q)
        sum += ct_resid(cl, v, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + (q >> 2));
      vc.b[e] = 0.5f * sum;
    }
    cl.sync();
  }
  {  // coarsest: x = Minv (-(b - mean b)) in FP64, rows spread over the cluster
    const CtView v(ct_smem, a.lv[last], rank);
    const int n = a.lv[last].n;
    float *gb = ct_smem + scratch;
    for (int e = threadIdx.x; e < n; e += CTL_THREADS) {
      const int k = ct_div(e, v.mpl);
      gb[e] = v.plane(cl, v.b, k)[e - k * v.pl];
    }
    __syncthreads();
    double acc0 = 0.0;
    for (int e = threadIdx.x; e < n; e += CTL_THREADS) acc0 += (double)gb[e];
    const double sum = block_sum(acc0);
    if (threadIdx.x == 0) mean_s = a.singular ? sum / n : 0.0;
    __syncthreads();
    const double m = mean_s;
    for (int r = rank * CTL_THREADS + threadIdx.x; r < n; r += CT_CTAS * CTL_THREADS) {
      double acc = 0.0;
      for (int c = 0; c < n; ++c) acc = fma(a.Minv[(size_t)c * n + r], (double)gb[c] - m, acc);
      const int k = ct_div(r, v.mpl);
      v.plane(cl, v.x, k)[r - k * v.pl] = (float)(-acc);
    }
    cl.sync();
  }
  for (int l = last - 1; l >= 0; --l) {  // up
    const CtView v(ct_smem, a.lv[l], rank), vc(ct_smem, a.lv[l + 1], rank);
    for (int e = threadIdx.x; e < v.own * v.pl; e += CTL_THREADS) {
      const int kq = ct_div(e, v.mpl), r = e - kq * v.pl, j = ct_div(r, v.mnx);
      const int i = r - j * v.nx, k = v.k0 + kq;
      v.x[e] += vc.plane(cl, vc.x, k >> 1)[(i >> 1) + vc.nx * (j >> 1)];
    }
    cl.sync();
    for (int s = 0; s < a.lv[l].nu2; ++s) {
      ct_halfsweep(cl, v, 1, 0);
      cl.sync();
      ct_halfsweep(cl, v, 0, 0);
      cl.sync();
    }
  }
  // (the last barrier above ends every access to another CTA's slab)
  const CtView v0(ct_smem, a.lv[0], rank);
  const size_t g0 = (size_t)v0.k0 * v0.pl;
  for (int e = threadIdx.x; e < v0.own * v0.pl; e += CTL_THREADS) xout[g0 + e] = v0.x[e];
}

}  // namespace mp
