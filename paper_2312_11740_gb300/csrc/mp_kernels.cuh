// Device kernels of the pressure-Poisson hot path (sm_103a).
//
// Conventions: cell arrays are C order, x fastest; face arrays use low-face
// ownership (element (i,j,k) of the x-face array is the face between cells
// i-1 and i, wrapped; on a wall axis face 0 is the wall and holds beta = 0).
// Inside the solver every level works with the h^2-scaled system
//   At e = bt,  (At e)_c = sum_f beta_f e_nb - diag_c e_c,  bt = h^2 b,
// so no kernel multiplies by 1/h^2; diag_c = sum of the six face betas.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mp {

struct Dims {
  int nx, ny, nz;
};

constexpr int BX = 32, BY = 8;  // per-cell launch tile (x fastest)

// First statement of the V-cycle kernels: they are launched with programmatic
// stream serialization (their blocks may be scheduled while the previous
// kernel finishes) and read nothing before the previous kernel has completed
// and its writes are visible.  A no-op for an ordinary launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ size_t at(const Dims &d, int i, int j, int k) {
  return (size_t)i + (size_t)d.nx * ((size_t)j + (size_t)d.ny * (size_t)k);
}
__device__ __forceinline__ int wlo(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int whi(int i, int n) { return i == n - 1 ? 0 : i + 1; }
// ghost index for one-sided stencils of phi: wrap on periodic axes, even
// mirror (ghost -1 -> 0, ghost n -> n-1) on wall axes
__device__ __forceinline__ int glo(int i, int n, bool per) { return i > 0 ? i - 1 : (per ? n - 1 : 0); }
__device__ __forceinline__ int ghi(int i, int n, bool per) { return i < n - 1 ? i + 1 : (per ? 0 : n - 1); }

// ---------------------------------------------------------------- reductions
template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order (deterministic for a fixed launch shape).
// Every thread must call it; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  int lane = (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) & 31;
  int warp = (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) >> 5;
  int nwarp = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < nwarp ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

__device__ __forceinline__ int block_linear_id() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ bool thread0() {
  return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
}

// phi > 0 (gas) tested on the bit pattern: an integer comparison instead of
// an FP64 one (FP64 instructions are the scarce resource of the setup kernels)
__device__ __forceinline__ bool gas(double v) { return __double_as_longlong(v) > 0; }

// ------------------------------------------------------------ A1: curvature
// kappa = -div(grad phi/|grad phi|) by central differences at cell centres,
// |grad phi| floored at 1e-12, |kappa| clamped to 1/h.  Gas-positive phi
// gives kappa = +2/R for a spherical bubble.  Only the jump across interface
// faces uses kappa, so it is evaluated in the interface band (cells with a
// face neighbour of the other fluid) and set to 0 elsewhere: FP64 division
// and square root are costly on this part, and the band is a thin shell.
__global__ void k_curvature(const double *__restrict__ phi, double *__restrict__ kap, Dims d,
                            double h, int per) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  bool px = per & 1, py = per & 2, pz = per & 4;
  int im = glo(i, d.nx, px), ip = ghi(i, d.nx, px);
  int jm = glo(j, d.ny, py), jp = ghi(j, d.ny, py);
  int km = glo(k, d.nz, pz), kp = ghi(k, d.nz, pz);
  double c = phi[at(d, i, j, k)];
  double xm = phi[at(d, im, j, k)], xp = phi[at(d, ip, j, k)];
  double ym = phi[at(d, i, jm, k)], yp = phi[at(d, i, jp, k)];
  double zm = phi[at(d, i, j, km)], zp = phi[at(d, i, j, kp)];
  bool gc = gas(c);
  bool band = (gas(xm) != gc) || (gas(xp) != gc) || (gas(ym) != gc) || (gas(yp) != gc) ||
              (gas(zm) != gc) || (gas(zp) != gc);
  if (!band) {
    kap[at(d, i, j, k)] = 0.0;
    return;
  }
  double i2h = 0.5 / h, ih2 = 1.0 / (h * h), i4h2 = 0.25 / (h * h);
  double gx = (xp - xm) * i2h, gy = (yp - ym) * i2h, gz = (zp - zm) * i2h;
  double gxx = (xp - 2.0 * c + xm) * ih2, gyy = (yp - 2.0 * c + ym) * ih2,
         gzz = (zp - 2.0 * c + zm) * ih2;
  double gxy = (phi[at(d, ip, jp, k)] - phi[at(d, ip, jm, k)] - phi[at(d, im, jp, k)] +
                phi[at(d, im, jm, k)]) * i4h2;
  double gxz = (phi[at(d, ip, j, kp)] - phi[at(d, ip, j, km)] - phi[at(d, im, j, kp)] +
                phi[at(d, im, j, km)]) * i4h2;
  double gyz = (phi[at(d, i, jp, kp)] - phi[at(d, i, jp, km)] - phi[at(d, i, jm, kp)] +
                phi[at(d, i, jm, km)]) * i4h2;
  double g = sqrt(gx * gx + gy * gy + gz * gz);
  g = g < 1e-12 ? 1e-12 : g;
  double num = gx * gx * (gyy + gzz) + gy * gy * (gxx + gzz) + gz * gz * (gxx + gyy) -
               2.0 * (gx * gy * gxy + gx * gz * gxz + gy * gz * gyz);
  double kv = -num / (g * g * g);
  double lim = 1.0 / h;
  kv = kv > lim ? lim : (kv < -lim ? -lim : kv);
  kap[at(d, i, j, k)] = kv;
}

// ------------------------------------------------- A2: ghost-fluid faces
// Two cells on one side: 1/rho of that fluid.  Across the interface the
// fluids act in series over the fractions theta, 1-theta of the spacing:
// beta = 1/(theta rho_a + (1-theta) rho_b), theta = |phi_a|/(|phi_a|+|phi_b|).
// irl = 1/rho_l and irg = 1/rho_g come from the host (the same IEEE quotient
// as computing 1/rho here), so single-fluid faces cost no division.
__device__ __forceinline__ double gfm_beta(double pa, double pb, double rl, double rg, double irl,
                                           double irg) {
  bool ga = gas(pa), gb = gas(pb);
  if (ga == gb) return ga ? irg : irl;
  double ra = ga ? rg : rl, rb = gb ? rg : rl;
  double th = fabs(pa) / (fabs(pa) + fabs(pb));
  return 1.0 / (th * ra + (1.0 - th) * rb);
}

// Pressure jump [p]_{a->b} = p(b side) - p(a side) = +-sigma kappa_G,
// kappa_G linearly interpolated to the interface; 0 off the interface.
__device__ __forceinline__ double gfm_jump(double pa, double pb, double ka, double kb, double sig) {
  bool ga = gas(pa), gb = gas(pb);
  if (ga == gb) return 0.0;
  double aa = fabs(pa), ab = fabs(pb);
  double kg = (ab * ka + aa * kb) / (aa + ab);
  return gb ? sig * kg : -sig * kg;
}

__global__ void k_faces(const double *__restrict__ phi, double *__restrict__ bx,
                        double *__restrict__ by, double *__restrict__ bz, Dims d, double rl,
                        double rg, double irl, double irg, int per) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  size_t c = at(d, i, j, k);
  double pc = phi[c];
  bx[c] = (i == 0 && !(per & 1)) ? 0.0
                                 : gfm_beta(phi[at(d, wlo(i, d.nx), j, k)], pc, rl, rg, irl, irg);
  by[c] = (j == 0 && !(per & 2)) ? 0.0
                                 : gfm_beta(phi[at(d, i, wlo(j, d.ny), k)], pc, rl, rg, irl, irg);
  bz[c] = (k == 0 && !(per & 4)) ? 0.0
                                 : gfm_beta(phi[at(d, i, j, wlo(k, d.nz))], pc, rl, rg, irl, irg);
}

// Phase change (evaporation): a liquid-to-gas mass flux mdot makes the
// normal velocity jump by mdot [1/rho], [1/rho] = 1/rho_g - 1/rho_l, so the
// pressure flux jumps by B = -mdot_G [1/rho] across an interface face, mdot_G
// interpolated to the interface point like the curvature.  Solving the two
// jump conditions with p linear on each side, the row of cell c takes the
// share beta theta_nb rho_nb B / h of a face to nb (theta_nb the fraction of
// the c-nb segment in nb's fluid); the two rows of a face take B / h in all.
__device__ __forceinline__ double flux_jump_B(double pa, double pb, double ma, double mb,
                                              double jinv) {
  const double aa = fabs(pa), ab = fabs(pb);
  return -((ab * ma + aa * mb) / (aa + ab)) * jinv;
}
// beta theta_nb rho_nb for the row of cell c (value pc) across a face to nb
__device__ __forceinline__ double flux_share(double pc, double pnb, double beta, double rl,
                                             double rg) {
  return beta * (fabs(pnb) / (fabs(pc) + fabs(pnb))) * (gas(pnb) ? rg : rl);
}

// -------------------------------------------------------- A3: jump source
// Flux across a face a->b is beta (p_b - p_a - [p]_{a->b}); moving the known
// jump to the right-hand side adds +beta [p]_{a->b} to row a and -beta
// [p]_{a->b} to row b.  Gathered per cell (no atomics); h^2-scaled.  With a
// mass flux (mdot not null) every interface face also adds the row's share
// of the flux jump (flux_share * B * h after the h^2 scaling).
__global__ void k_jump(const double *__restrict__ phi, const double *__restrict__ kap,
                       const double *__restrict__ bx, const double *__restrict__ by,
                       const double *__restrict__ bz, double *__restrict__ Jt, Dims d,
                       double sig, const double *__restrict__ mdot, double rl, double rg,
                       double h) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  size_t c = at(d, i, j, k);
  double pc = phi[c];
  size_t xl = at(d, wlo(i, d.nx), j, k), xh = at(d, whi(i, d.nx), j, k);
  size_t yl = at(d, i, wlo(j, d.ny), k), yh = at(d, i, whi(j, d.ny), k);
  size_t zl = at(d, i, j, wlo(k, d.nz)), zh = at(d, i, j, whi(k, d.nz));
  const bool g = gas(pc);
  if (gas(phi[xl]) == g && gas(phi[xh]) == g && gas(phi[yl]) == g && gas(phi[yh]) == g &&
      gas(phi[zl]) == g && gas(phi[zh]) == g) {
    Jt[c] = 0.0;  // no interface on any face of the cell
    return;
  }
  double kc = kap[c];
  double s = 0.0;
  s += bx[xh] * gfm_jump(pc, phi[xh], kc, kap[xh], sig) - bx[c] * gfm_jump(phi[xl], pc, kap[xl], kc, sig);
  s += by[yh] * gfm_jump(pc, phi[yh], kc, kap[yh], sig) - by[c] * gfm_jump(phi[yl], pc, kap[yl], kc, sig);
  s += bz[zh] * gfm_jump(pc, phi[zh], kc, kap[zh], sig) - bz[c] * gfm_jump(phi[zl], pc, kap[zl], kc, sig);
  if (mdot) {
    const double jinv = 1.0 / rg - 1.0 / rl, mc = mdot[c];
    const size_t nb[6] = {xl, xh, yl, yh, zl, zh};
    const double bf[6] = {bx[c], bx[xh], by[c], by[yh], bz[c], bz[zh]};
    double f = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double pn = phi[nb[q]];
      if (gas(pn) == g || bf[q] == 0.0) continue;  // no interface, or a wall face
      f += flux_share(pc, pn, bf[q], rl, rg) * flux_jump_B(pc, pn, mc, mdot[nb[q]], jinv);
    }
    s = fma(f, h, s);
  }
  Jt[c] = s;
}

// Outflow boundary sides of a level: per side (x low, x high, y low, y
// high, z low, z high) the coefficients of the boundary faces as a plane
// (x sides: j + ny k; y sides: i + nx k; z sides: i + nx j), or null.
struct BndPlanes {
  const double *p[6];
};
// 2 beta_b summed over the outflow faces of cell (i, j, k): the ghost value
// -x_c turns a face's term beta_b (x_ghost - x_c) into -2 beta_b x_c
__device__ __forceinline__ double outflow_diag(const BndPlanes &bp, const Dims &d, int i, int j,
                                               int k) {
  double s = 0.0;
  if (i == 0 && bp.p[0]) s += 2.0 * bp.p[0][j + d.ny * k];
  if (i == d.nx - 1 && bp.p[1]) s += 2.0 * bp.p[1][j + d.ny * k];
  if (j == 0 && bp.p[2]) s += 2.0 * bp.p[2][i + d.nx * k];
  if (j == d.ny - 1 && bp.p[3]) s += 2.0 * bp.p[3][i + d.nx * k];
  if (k == 0 && bp.p[4]) s += 2.0 * bp.p[4][i + d.nx * j];
  if (k == d.nz - 1 && bp.p[5]) s += 2.0 * bp.p[5][i + d.nx * j];
  return s;
}

// diag = sum of the six face betas (always), plus the outflow diagonal when
// dd is not null (stored in dd, and as FP32 / scaled FP16 copies with MODE
// & 2); MODE & 1: idiag = 1/diag (the FP64 smoother); MODE & 2: FP32 faces
// and 1/diag (CG operator, one-CTA tail) and the FP16 faces of the FP32
// V-cycle, stored as beta * fs
template <int MODE>
__global__ void k_diag(const double *__restrict__ bx, const double *__restrict__ by,
                       const double *__restrict__ bz, double *__restrict__ diag,
                       double *__restrict__ idiag, float *__restrict__ bx32,
                       float *__restrict__ by32, float *__restrict__ bz32,
                       float *__restrict__ idiag32, __half *__restrict__ bx16,
                       __half *__restrict__ by16, __half *__restrict__ bz16, float fs, Dims d,
                       BndPlanes bp, double *__restrict__ dd, float *__restrict__ dd32,
                       __half *__restrict__ dd16) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  size_t c = at(d, i, j, k);
  double s = bx[c] + bx[at(d, whi(i, d.nx), j, k)] + by[c] + by[at(d, i, whi(j, d.ny), k)] + bz[c] +
             bz[at(d, i, j, whi(k, d.nz))];
  if (dd) {
    const double o = outflow_diag(bp, d, i, j, k);
    dd[c] = o;
    s += o;
    if (MODE & 2) {
      dd32[c] = (float)o;
      dd16[c] = __float2half_rn((float)o * fs * 0.25f);  // see dd_h
    }
  }
  diag[c] = s;
  if (MODE & 1) {
    // 1/s: FP32 reciprocal refined by one Newton step in FP64 (relative error
    // ~1e-14, two FP64 operations instead of a full FP64 division)
    double is = (double)(1.0f / (float)s);
    is = is * fma(-s, is, 2.0);
    idiag[c] = is;
  }
  if (MODE & 2) {
    const float fx = (float)bx[c], fy = (float)by[c], fz = (float)bz[c];
    bx32[c] = fx;
    by32[c] = fy;
    bz32[c] = fz;
    idiag32[c] = 1.0f / (float)s;
    bx16[c] = __float2half_rn(fx * fs);
    by16[c] = __float2half_rn(fy * fs);
    bz16[c] = __float2half_rn(fz * fs);
  }
}

// ------------------------------------------- A5: coarse face coefficients
// A coarse face is the mean of the four fine faces that tile it.
__global__ void k_coarsen_faces(const double *__restrict__ fx, const double *__restrict__ fy,
                                const double *__restrict__ fz, Dims df, double *__restrict__ cx,
                                double *__restrict__ cy, double *__restrict__ cz, Dims dc) {
  int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (I >= dc.nx || J >= dc.ny) return;
  int i = 2 * I, j = 2 * J, k = 2 * K;
  size_t c = at(dc, I, J, K);
  cx[c] = 0.25 * (fx[at(df, i, j, k)] + fx[at(df, i, j + 1, k)] + fx[at(df, i, j, k + 1)] +
                  fx[at(df, i, j + 1, k + 1)]);
  cy[c] = 0.25 * (fy[at(df, i, j, k)] + fy[at(df, i + 1, j, k)] + fy[at(df, i, j, k + 1)] +
                  fy[at(df, i + 1, j, k + 1)]);
  cz[c] = 0.25 * (fz[at(df, i, j, k)] + fz[at(df, i + 1, j, k)] + fz[at(df, i, j + 1, k)] +
                  fz[at(df, i + 1, j + 1, k)]);
}

// ---------------------------------------------- A9: coarsest direct solve
// Dense M = -At + 11^T/n (symmetric positive definite; the 11^T/n term only
// for a singular operator) as the left half of [M | I] (row-major, n x 2n);
// one thread per row, each row written once.
__global__ void k_dense_build(const double *__restrict__ bx, const double *__restrict__ by,
                              const double *__restrict__ bz, const double *__restrict__ diag,
                              double *__restrict__ M, Dims d, int singular) {
  int n = d.nx * d.ny * d.nz;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int i = r % d.nx, j = (r / d.nx) % d.ny, k = r / (d.nx * d.ny);
  double *row = M + (size_t)r * 2 * n;
  double inv_n = singular ? 1.0 / n : 0.0;
  for (int c = 0; c < n; ++c) row[c] = inv_n;
  for (int c = 0; c < n; ++c) row[n + c] = (c == r) ? 1.0 : 0.0;
  row[r] += diag[r];
  row[at(d, wlo(i, d.nx), j, k)] -= bx[r];
  row[at(d, whi(i, d.nx), j, k)] -= bx[at(d, whi(i, d.nx), j, k)];
  row[at(d, i, wlo(j, d.ny), k)] -= by[r];
  row[at(d, i, whi(j, d.ny), k)] -= by[at(d, i, whi(j, d.ny), k)];
  row[at(d, i, j, wlo(k, d.nz))] -= bz[r];
  row[at(d, i, j, whi(k, d.nz))] -= bz[at(d, i, j, whi(k, d.nz))];
}

// Gauss-Jordan elimination of [M | I] -> [I | M^-1] by one block (M is SPD,
// so no pivoting).  n <= 512.  The inverse (symmetric) is copied to Minv.
__global__ void k_gauss_jordan(double *__restrict__ M, double *__restrict__ Minv, int n) {
  __shared__ double col[512];
  const int w = 2 * n;
  for (int p = 0; p < n; ++p) {
    for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = M[(size_t)r * w + p];
    __syncthreads();
    double inv = 1.0 / col[p];
    for (int c = threadIdx.x; c < w; c += blockDim.x) M[(size_t)p * w + c] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
      int r = e / w, c = e - r * w;
      if (r != p) M[(size_t)r * w + c] -= col[r] * M[(size_t)p * w + c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    Minv[e] = M[(size_t)r * w + n + c];
  }
}

// Inverse of the SPD coarsest matrix M (left half of [M | I]) by columns, for
// n <= GJ_SMEM_MAX: block j factors M = L L^T in shared memory (every block the
// same factor) and solves L L^T x = e_j into column j.  The n blocks run on n
// SMs at once; one block's Gauss-Jordan elimination is bound by a single SM's
// FP64 rate, which is low on this part.
constexpr int GJ_SMEM_MAX = 112;
__global__ void k_inverse_cols(const double *__restrict__ Maug, double *__restrict__ Minv, int n) {
  extern __shared__ double L[];  // n x n, then the right-hand side / solution (n)
  __shared__ double inv_d[GJ_SMEM_MAX];
  double *y = L + n * n;
  const int w = 2 * n, j = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) L[e] = Maug[(size_t)(e / n) * w + (e % n)];
  for (int e = tid; e < n; e += nt) y[e] = e == j ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {  // right-looking Cholesky, lower triangle
    if (tid == 0) {
      const double dkk = sqrt(L[k * n + k]);
      L[k * n + k] = dkk;
      inv_d[k] = 1.0 / dkk;
    }
    __syncthreads();
    const double id = inv_d[k];
    for (int r = k + 1 + tid; r < n; r += nt) L[r * n + k] *= id;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int r = k + 1 + e / m, c = k + 1 + e % m;
      if (c <= r) L[r * n + c] -= L[r * n + k] * L[c * n + k];
    }
    __syncthreads();
  }
  for (int c = 0; c < n; ++c) {  // L y = e_j (column-oriented)
    if (tid == 0) y[c] *= inv_d[c];
    __syncthreads();
    for (int r = c + 1 + tid; r < n; r += nt) y[r] -= L[r * n + c] * y[c];
    __syncthreads();
  }
  for (int c = n - 1; c >= 0; --c) {  // L^T x = y
    if (tid == 0) y[c] *= inv_d[c];
    __syncthreads();
    for (int r = tid; r < c; r += nt) y[r] -= L[c * n + r] * y[c];
    __syncthreads();
  }
  for (int r = tid; r < n; r += nt) Minv[(size_t)r * n + j] = y[r];
}

// e = M^-1 (-(b - mean b)), FP64 internally for any storage type T (the
// mean is removed only for a singular operator).  One block of 512
// threads; n <= 512.
template <typename T>
__global__ void k_coarse_solve(const double *__restrict__ Minv, const T *__restrict__ b,
                               T *__restrict__ e, int n, int singular) {
  griddep_wait();
  __shared__ double sb[512];
  __shared__ double mean;
  int t = threadIdx.x;
  double v = t < n ? (double)b[t] : 0.0;
  double s = block_sum(v);
  if (t == 0) mean = singular ? s / n : 0.0;
  __syncthreads();
  sb[t] = t < n ? v - mean : 0.0;
  __syncthreads();
  if (t < n) {
    double acc = 0.0;
    for (int c = 0; c < n; ++c) acc = fma(Minv[(size_t)c * n + t], sb[c], acc);
    e[t] = (T)(-acc);
  }
}

// ------------------------------------------------- A6: red-black smoother
// One colour ((i+j+k) & 1 == colour): x_c = (sum_f beta_f x_nb - bt_c) / diag_c,
// in place (a colour's update reads only the other colour).  zero != 0
// treats x as zero before the update (first sweep of a cycle).
template <typename T>
__device__ __forceinline__ void rbgs_cell(T *__restrict__ x, const T *__restrict__ b,
                                          const T *__restrict__ bx, const T *__restrict__ by,
                                          const T *__restrict__ bz, const T *__restrict__ idiag,
                                          const Dims &d, int t, int j, int k, int colour,
                                          int zero) {
  int i = 2 * t + ((j + k + colour) & 1);
  size_t c = at(d, i, j, k);
  size_t xl = at(d, wlo(i, d.nx), j, k), xh = at(d, whi(i, d.nx), j, k);
  size_t yl = at(d, i, wlo(j, d.ny), k), yh = at(d, i, whi(j, d.ny), k);
  size_t zl = at(d, i, j, wlo(k, d.nz)), zh = at(d, i, j, whi(k, d.nz));
  const T wxl = bx[c], wxh = bx[xh], wyl = by[c], wyh = by[yh], wzl = bz[c], wzh = bz[zh];
  T s = -b[c];
  if (!zero) {
    s = fma(wxl, x[xl], s);
    s = fma(wxh, x[xh], s);
    s = fma(wyl, x[yl], s);
    s = fma(wyh, x[yh], s);
    s = fma(wzl, x[zl], s);
    s = fma(wzh, x[zh], s);
  }
  if (sizeof(T) == 8) {
    x[c] = s * idiag[c];  // stored 1/diag: no FP64 division
  } else {
    x[c] = __fdividef((float)s, (float)(((wxl + wxh) + (wyl + wyh)) + (wzl + wzh)));
  }
}

template <typename T>
__global__ void k_rbgs(T *__restrict__ x, const T *__restrict__ b, const T *__restrict__ bx,
                       const T *__restrict__ by, const T *__restrict__ bz,
                       const T *__restrict__ idiag, Dims d, int colour, int zero) {
  griddep_wait();
  int t = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (t >= (d.nx >> 1) || j >= d.ny) return;
  rbgs_cell<T>(x, b, bx, by, bz, idiag, d, t, j, k, colour, zero);
}

// (At x)_c at one cell.  FP64: sum_f beta_f x_nb - diag_c x_c (fewest FP64
// operations; FP64 keeps ~13 digits after the cancellation at density
// ratio 1e3).  FP32: sum_f beta_f (x_nb - x_c): differences first, so the
// cancellation between the beta ~ 1e3 terms of a gas cell does not eat the
// 7-digit FP32 mantissa.  dd (may be null): the diagonal of the outflow
// faces of the cell (2 beta_b per outflow face: the ghost value -x_c),
// subtracted in the difference form (the stored diag already holds it).
template <typename T>
__device__ __forceinline__ T op_at(const T *__restrict__ x, const T *__restrict__ bx,
                                   const T *__restrict__ by, const T *__restrict__ bz,
                                   const T *__restrict__ diag, const T *__restrict__ dd,
                                   const Dims &d, int i, int j, int k) {
  size_t c = at(d, i, j, k);
  size_t xl = at(d, wlo(i, d.nx), j, k), xh = at(d, whi(i, d.nx), j, k);
  size_t yl = at(d, i, wlo(j, d.ny), k), yh = at(d, i, whi(j, d.ny), k);
  size_t zl = at(d, i, j, wlo(k, d.nz)), zh = at(d, i, j, whi(k, d.nz));
  T xc = x[c];
  if (sizeof(T) == 8 && diag != nullptr) {
    T s = -diag[c] * xc;
    s = fma(bx[c], x[xl], s);
    s = fma(bx[xh], x[xh], s);
    s = fma(by[c], x[yl], s);
    s = fma(by[yh], x[yh], s);
    s = fma(bz[c], x[zl], s);
    s = fma(bz[zh], x[zh], s);
    return s;
  } else {
    T s = bx[c] * (x[xl] - xc);
    s = fma(bx[xh], x[xh] - xc, s);
    s = fma(by[c], x[yl] - xc, s);
    s = fma(by[yh], x[yh] - xc, s);
    s = fma(bz[c], x[zl] - xc, s);
    s = fma(bz[zh], x[zh] - xc, s);
    if (dd) s = fma(-dd[c], xc, s);
    return s;
  }
}

// scaled residual at one cell: rt = bt - (At x)_c
template <typename T>
__device__ __forceinline__ T resid_at(const T *__restrict__ x, const T *__restrict__ b,
                                      const T *__restrict__ bx, const T *__restrict__ by,
                                      const T *__restrict__ bz, const T *__restrict__ diag,
                                      const T *__restrict__ dd, const Dims &d, int i, int j,
                                      int k) {
  return b[at(d, i, j, k)] - op_at(x, bx, by, bz, diag, dd, d, i, j, k);
}


// ------------------------------------------ A6-A9: coarse tail in one CTA
// The bottom of the V-cycle (levels of at most a few thousand cells) in a
// single launch: every level's iterate, right-hand side and face
// coefficients live in shared memory, and one 1024-thread block runs all
// sweeps, restrictions, prolongations and the FP64 coarsest solve with
// __syncthreads between steps.  Replaces ~100 latency-bound launches per
// cycle.  Same arithmetic as the per-level kernels (colour order, difference
// form for FP32 residuals, diag formed from the faces).
constexpr int TAIL_MAX_LEVELS = 8;
constexpr int TAIL_THREADS = 1024;
struct TailLevel {
  Dims d;
  int n, nu1, nu2;
  int off;  // element offset of the level's arrays in shared memory
  const void *bx, *by, *bz, *idiag;
  const void *dd;  // outflow diagonal (null without outflow sides)
};
struct TailArgs {
  int nlev;  // levels in the tail (the last one is the coarsest)
  TailLevel lv[TAIL_MAX_LEVELS];
  const double *Minv;
  int singular;  // the operator annihilates constants: mean-project the coarsest rhs
};

// shared-memory arrays of one tail level: x, b, bx, by, bz, 1/diag, and the
// outflow diagonal when the level has one
template <typename T>
struct TailView {
  T *x, *b, *wx, *wy, *wz, *id, *dd;
  __device__ TailView(T *base, const TailLevel &l) {
    x = base + l.off;
    b = x + l.n;
    wx = b + l.n;
    wy = wx + l.n;
    wz = wy + l.n;
    id = wz + l.n;
    dd = l.dd ? id + l.n : nullptr;
  }
};

template <typename T>
__device__ __forceinline__ void tail_halfsweep(const TailView<T> &v, const Dims &d, int colour,
                                               int zero) {
  const int nx = d.nx, ny = d.ny, nz = d.nz, sy = nx, sz = nx * ny;
  const int hx = nx >> 1, half = (nx * ny * nz) >> 1;
  for (int t = threadIdx.x; t < half; t += TAIL_THREADS) {
    const int row = t / hx;
    const int j = row % ny, k = row / ny;
    const int i = 2 * (t - row * hx) + ((j + k + colour) & 1);
    const int c = i + j * sy + k * sz;
    const int xp = i == nx - 1 ? c - (nx - 1) : c + 1;
    const int yp = j == ny - 1 ? c - (ny - 1) * sy : c + sy;
    const int zp = k == nz - 1 ? c - (nz - 1) * sz : c + sz;
    T num = -v.b[c];
    if (!zero) {
      const int xm = i == 0 ? c + (nx - 1) : c - 1;
      const int ym = j == 0 ? c + (ny - 1) * sy : c - sy;
      const int zm = k == 0 ? c + (nz - 1) * sz : c - sz;
      num = fma(v.wx[c], v.x[xm], num);
      num = fma(v.wx[xp], v.x[xp], num);
      num = fma(v.wy[c], v.x[ym], num);
      num = fma(v.wy[yp], v.x[yp], num);
      num = fma(v.wz[c], v.x[zm], num);
      num = fma(v.wz[zp], v.x[zp], num);
    }
    v.x[c] = num * v.id[c];
  }
}

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS)
k_tail(TailArgs a, const T *__restrict__ rhs, T *__restrict__ xout) {
  griddep_wait();
  extern __shared__ __align__(16) unsigned char tail_smem[];
  T *base = reinterpret_cast<T *>(tail_smem);
  for (int l = 0; l < a.nlev; ++l) {
    TailView<T> v(base, a.lv[l]);
    const T *gx = (const T *)a.lv[l].bx, *gy = (const T *)a.lv[l].by, *gz = (const T *)a.lv[l].bz,
            *gi = (const T *)a.lv[l].idiag;
    const T *gd = (const T *)a.lv[l].dd;
    for (int e = threadIdx.x; e < a.lv[l].n; e += TAIL_THREADS) {
      v.wx[e] = gx[e];
      v.wy[e] = gy[e];
      v.wz[e] = gz[e];
      v.id[e] = gi[e];
      if (gd) v.dd[e] = gd[e];
    }
  }
  {
    TailView<T> v0(base, a.lv[0]);
    for (int e = threadIdx.x; e < a.lv[0].n; e += TAIL_THREADS) v0.b[e] = rhs[e];
  }
  __syncthreads();
  const int last = a.nlev - 1;
  for (int l = 0; l < last; ++l) {  // down
    const TailView<T> v(base, a.lv[l]);
    const TailView<T> vc(base, a.lv[l + 1]);
    const Dims d = a.lv[l].d, dc = a.lv[l + 1].d;
    for (int s = 0; s < a.lv[l].nu1; ++s) {
      tail_halfsweep(v, d, 0, s == 0);
      __syncthreads();
      tail_halfsweep(v, d, 1, 0);
      __syncthreads();
    }
    for (int e = threadIdx.x; e < a.lv[l + 1].n; e += TAIL_THREADS) {
      const int I = e % dc.nx, J = (e / dc.nx) % dc.ny, K = e / (dc.nx * dc.ny);
      T sum = 0;
      for (int q = 0; q < 8; ++q)
        sum += resid_at(v.x, v.b, v.wx, v.wy, v.wz, (const T *)nullptr, (const T *)v.dd, d,
                        2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + (q >> 2));
      vc.b[e] = (T)0.5 * sum;
    }
    __syncthreads();
  }
  {  // coarsest: e = Minv (-(b - mean b)) in FP64
    __shared__ double mean_s;
    const TailView<T> v(base, a.lv[last]);
    const int n = a.lv[last].n;
    double acc0 = 0.0;
    for (int e = threadIdx.x; e < n; e += TAIL_THREADS) acc0 += (double)v.b[e];
    double sum = block_sum(acc0);
    if (threadIdx.x == 0) mean_s = a.singular ? sum / n : 0.0;
    __syncthreads();
    const double m = mean_s;
    for (int r = threadIdx.x; r < n; r += TAIL_THREADS) {
      double acc = 0.0;
      for (int c = 0; c < n; ++c) acc = fma(a.Minv[(size_t)c * n + r], (double)v.b[c] - m, acc);
      v.x[r] = (T)(-acc);
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {  // up
    const TailView<T> v(base, a.lv[l]);
    const TailView<T> vc(base, a.lv[l + 1]);
    const Dims d = a.lv[l].d, dc = a.lv[l + 1].d;
    for (int e = threadIdx.x; e < a.lv[l].n; e += TAIL_THREADS) {
      const int i = e % d.nx, j = (e / d.nx) % d.ny, k = e / (d.nx * d.ny);
      v.x[e] += vc.x[(i >> 1) + dc.nx * ((j >> 1) + dc.ny * (k >> 1))];
    }
    __syncthreads();
    for (int s = 0; s < a.lv[l].nu2; ++s) {
      tail_halfsweep(v, d, 1, 0);
      __syncthreads();
      tail_halfsweep(v, d, 0, 0);
      __syncthreads();
    }
  }
  const TailView<T> v0(base, a.lv[0]);
  for (int e = threadIdx.x; e < a.lv[0].n; e += TAIL_THREADS) xout[e] = v0.x[e];
}

// ------------------------------------- A7: residual + restriction (fused)
// Coarse scaled rhs = (2h)^2 * mean of the 8 children's residuals
//                   = 0.5 * sum of the children's scaled residuals.
template <typename T>
__device__ __forceinline__ void resid_restrict_cell(const T *__restrict__ x,
                                                    const T *__restrict__ b,
                                                    const T *__restrict__ bx,
                                                    const T *__restrict__ by,
                                                    const T *__restrict__ bz,
                                                    const T *__restrict__ diag, const Dims &df,
                                                    T *__restrict__ bc, const Dims &dc, int I,
                                                    int J, int K) {
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    s += resid_at(x, b, bx, by, bz, diag, (const T *)nullptr, df, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1),
                  2 * K + (q >> 2));
  bc[at(dc, I, J, K)] = (T)0.5 * s;
}

// ------------------------- FP32 V-cycle sweeps on FP16 face coefficients
// The finest levels of the FP32 V-cycle read their face coefficients as FP16
// copies scaled by a power of two fs (the largest coefficient lands just below
// 2^14, the smallest of a 1e8 density ratio stays a normal number): 6 instead
// of 12 bytes of coefficients per cell, the largest stream of a half-sweep.
// FP16 keeps 11 bits; the V-cycle is only the preconditioner, and its smoother
// and residual/restriction use the same rounded coefficients on every level
// they run on, so it stays one fixed symmetric operator.  The CG operator and
// every true residual keep the FP32/FP64 faces.
__device__ __forceinline__ float hf(const __half *__restrict__ p, size_t i) {
  return __half2float(p[i]);
}

// new value of one cell of a red-black half-sweep (loads only):
// x_c = (sum_f w_f x_nb - fs bt_c) / sum_f w_f with w = fs beta
// The FP16 outflow diagonal is stored as fs/4 times its value: up to six
// outflow faces of 2 beta fs <= 2^15 each stay below the FP16 maximum; the
// power-of-two factor is exact.
__device__ __forceinline__ float dd_h(const __half *__restrict__ dd16, size_t c) {
  return 4.f * __half2float(dd16[c]);
}

__device__ __forceinline__ float rbgs_h_val(const float *__restrict__ x,
                                            const float *__restrict__ b,
                                            const __half *__restrict__ hx,
                                            const __half *__restrict__ hy,
                                            const __half *__restrict__ hz,
                                            const __half *__restrict__ dd16, const Dims &d, int i,
                                            int j, int k, int zero, float fs) {
  const size_t c = at(d, i, j, k);
  const size_t xl = at(d, wlo(i, d.nx), j, k), xh = at(d, whi(i, d.nx), j, k);
  const size_t yl = at(d, i, wlo(j, d.ny), k), yh = at(d, i, whi(j, d.ny), k);
  const size_t zl = at(d, i, j, wlo(k, d.nz)), zh = at(d, i, j, whi(k, d.nz));
  const float wxl = hf(hx, c), wxh = hf(hx, xh), wyl = hf(hy, c), wyh = hf(hy, yh),
              wzl = hf(hz, c), wzh = hf(hz, zh);
  float s = -b[c] * fs;
  if (!zero) {
    s = fmaf(wxl, x[xl], s);
    s = fmaf(wxh, x[xh], s);
    s = fmaf(wyl, x[yl], s);
    s = fmaf(wyh, x[yh], s);
    s = fmaf(wzl, x[zl], s);
    s = fmaf(wzh, x[zh], s);
  }
  float den = ((wxl + wxh) + (wyl + wyh)) + (wzl + wzh);
  if (dd16) den += dd_h(dd16, c);
  return __fdividef(s, den);
}

// red-black half-sweep on the FP16 faces (one cell of the colour per thread;
// two planes per thread measured slower: fewer resident warps); dd16: the
// outflow diagonal scaled by fs, or null
__global__ void k_rbgs_h(float *__restrict__ x, const float *__restrict__ b,
                         const __half *__restrict__ hx, const __half *__restrict__ hy,
                         const __half *__restrict__ hz, const __half *__restrict__ dd16, Dims d,
                         int colour, int zero, float fs) {
  griddep_wait();
  const int t = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (t >= (d.nx >> 1) || j >= d.ny) return;
  const int i = 2 * t + ((j + k + colour) & 1);
  x[at(d, i, j, k)] = rbgs_h_val(x, b, hx, hy, hz, dd16, d, i, j, k, zero, fs);
}

// The same half-sweep with 16-byte rows (nx a multiple of 4, 16-byte aligned
// x and b): a thread owns the 4-cell x-chunk [4q, 4q + 4) of a row and
// updates its two cells of the colour, loading x, b and the faces of the
// chunk as vectors (14 loads for two cells instead of 26).  Each cell's
// arithmetic is that of rbgs_h_val, operation for operation in the same order.
struct __align__(8) H4 {
  __half2 a, b;
};
__device__ __forceinline__ float h4_at(const H4 &v, int q) {
  const __half2 p = q < 2 ? v.a : v.b;
  return (q & 1) ? __high2float(p) : __low2float(p);
}
__device__ __forceinline__ float f4_at(const float4 &v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

__global__ void k_rbgs_h4(float *__restrict__ x, const float *__restrict__ b,
                          const __half *__restrict__ hx, const __half *__restrict__ hy,
                          const __half *__restrict__ hz, const __half *__restrict__ dd16, Dims d,
                          int colour, int zero, float fs) {
  griddep_wait();
  const int qx = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (qx >= (d.nx >> 2) || j >= d.ny) return;
  const int i0 = 4 * qx;
  const int o = (j + k + colour) & 1;  // the chunk's cells of the colour: i0 + o, i0 + o + 2
  const size_t c0 = at(d, i0, j, k);
  const size_t cyl = at(d, i0, wlo(j, d.ny), k), cyh = at(d, i0, whi(j, d.ny), k);
  const size_t czl = at(d, i0, j, wlo(k, d.nz)), czh = at(d, i0, j, whi(k, d.nz));
  const float4 bb = *reinterpret_cast<const float4 *>(b + c0);
  const H4 fx = *reinterpret_cast<const H4 *>(hx + c0);
  const H4 fy = *reinterpret_cast<const H4 *>(hy + c0);
  const H4 fyh = *reinterpret_cast<const H4 *>(hy + cyh);
  const H4 fz = *reinterpret_cast<const H4 *>(hz + c0);
  const H4 fzh = *reinterpret_cast<const H4 *>(hz + czh);
  const float fxe = hf(hx, at(d, whi(i0 + 3, d.nx), j, k));  // high x face of cell i0 + 3
  float4 xc = make_float4(0.f, 0.f, 0.f, 0.f), xyl = xc, xyh = xc, xzl = xc, xzh = xc;
  float xm = 0.f, xp = 0.f;  // x[i0 - 1], x[i0 + 4] (wrapped)
  if (!zero) {
    xc = *reinterpret_cast<const float4 *>(x + c0);
    xyl = *reinterpret_cast<const float4 *>(x + cyl);
    xyh = *reinterpret_cast<const float4 *>(x + cyh);
    xzl = *reinterpret_cast<const float4 *>(x + czl);
    xzh = *reinterpret_cast<const float4 *>(x + czh);
    xm = x[at(d, wlo(i0, d.nx), j, k)];
    xp = x[at(d, whi(i0 + 3, d.nx), j, k)];
  }
  float v[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int q = o + 2 * e;  // position in the chunk
    const float wxl = h4_at(fx, q), wxh = q < 3 ? h4_at(fx, q + 1) : fxe;
    const float wyl = h4_at(fy, q), wyh = h4_at(fyh, q), wzl = h4_at(fz, q),
                wzh = h4_at(fzh, q);
    float s = -f4_at(bb, q) * fs;
    if (!zero) {
      const float x_l = q > 0 ? f4_at(xc, q - 1) : xm, x_h = q < 3 ? f4_at(xc, q + 1) : xp;
      s = fmaf(wxl, x_l, s);
      s = fmaf(wxh, x_h, s);
      s = fmaf(wyl, f4_at(xyl, q), s);
      s = fmaf(wyh, f4_at(xyh, q), s);
      s = fmaf(wzl, f4_at(xzl, q), s);
      s = fmaf(wzh, f4_at(xzh, q), s);
    }
    float den = ((wxl + wxh) + (wyl + wyh)) + (wzl + wzh);
    if (dd16) den += dd_h(dd16, c0 + q);
    v[e] = __fdividef(s, den);
  }
  x[c0 + o] = v[0];
  x[c0 + o + 2] = v[1];
}

// bt_c - (At x)_c with the FP16 faces (difference form, as the FP32 operator)
__device__ __forceinline__ float resid_h(const float *__restrict__ x, const float *__restrict__ b,
                                         const __half *__restrict__ hx,
                                         const __half *__restrict__ hy,
                                         const __half *__restrict__ hz,
                                         const __half *__restrict__ dd16, float inv_fs,
                                         const Dims &d, int i, int j, int k) {
  const size_t c = at(d, i, j, k);
  const size_t xl = at(d, wlo(i, d.nx), j, k), xh = at(d, whi(i, d.nx), j, k);
  const size_t yl = at(d, i, wlo(j, d.ny), k), yh = at(d, i, whi(j, d.ny), k);
  const size_t zl = at(d, i, j, wlo(k, d.nz)), zh = at(d, i, j, whi(k, d.nz));
  const float xc = x[c];
  float s = hf(hx, c) * (x[xl] - xc);
  s = fmaf(hf(hx, xh), x[xh] - xc, s);
  s = fmaf(hf(hy, c), x[yl] - xc, s);
  s = fmaf(hf(hy, yh), x[yh] - xc, s);
  s = fmaf(hf(hz, c), x[zl] - xc, s);
  s = fmaf(hf(hz, zh), x[zh] - xc, s);
  if (dd16) s = fmaf(-dd_h(dd16, c), xc, s);
  return b[c] - s * inv_fs;
}

// residual + restriction (half the sum of the 8 children) on the FP16 faces
__global__ void k_resid_restrict_h(const float *__restrict__ x, const float *__restrict__ b,
                                   const __half *__restrict__ hx, const __half *__restrict__ hy,
                                   const __half *__restrict__ hz, const __half *__restrict__ dd16,
                                   float inv_fs, Dims df, float *__restrict__ bc, Dims dc) {
  griddep_wait();
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (I >= dc.nx || J >= dc.ny) return;
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    s += resid_h(x, b, hx, hy, hz, dd16, inv_fs, df, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1),
                 2 * K + (q >> 2));
  bc[at(dc, I, J, K)] = 0.5f * s;
}

// Residuals bt - At x of the 4-cell x-chunk [i0, i0 + 4) of fine row (j, k),
// with the FP16 faces and 16-byte loads (resid_h's arithmetic per cell)
__device__ __forceinline__ void resid_h4(const float *__restrict__ x, const float *__restrict__ b,
                                         const __half *__restrict__ hx,
                                         const __half *__restrict__ hy,
                                         const __half *__restrict__ hz,
                                         const __half *__restrict__ dd16, float inv_fs,
                                         const Dims &d, int i0, int j, int k, float r[4]) {
  const size_t c0 = at(d, i0, j, k);
  const size_t cyl = at(d, i0, wlo(j, d.ny), k), cyh = at(d, i0, whi(j, d.ny), k);
  const size_t czl = at(d, i0, j, wlo(k, d.nz)), czh = at(d, i0, j, whi(k, d.nz));
  const float4 bb = *reinterpret_cast<const float4 *>(b + c0);
  const float4 xc = *reinterpret_cast<const float4 *>(x + c0);
  const float4 xyl = *reinterpret_cast<const float4 *>(x + cyl);
  const float4 xyh = *reinterpret_cast<const float4 *>(x + cyh);
  const float4 xzl = *reinterpret_cast<const float4 *>(x + czl);
  const float4 xzh = *reinterpret_cast<const float4 *>(x + czh);
  const H4 fx = *reinterpret_cast<const H4 *>(hx + c0);
  const H4 fy = *reinterpret_cast<const H4 *>(hy + c0);
  const H4 fyh = *reinterpret_cast<const H4 *>(hy + cyh);
  const H4 fz = *reinterpret_cast<const H4 *>(hz + c0);
  const H4 fzh = *reinterpret_cast<const H4 *>(hz + czh);
  const size_t ce = at(d, whi(i0 + 3, d.nx), j, k);
  const float fxe = hf(hx, ce), xp = x[ce], xm = x[at(d, wlo(i0, d.nx), j, k)];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float v = f4_at(xc, q);
    const float x_l = q > 0 ? f4_at(xc, q - 1) : xm, x_h = q < 3 ? f4_at(xc, q + 1) : xp;
    float s = h4_at(fx, q) * (x_l - v);
    s = fmaf(q < 3 ? h4_at(fx, q + 1) : fxe, x_h - v, s);
    s = fmaf(h4_at(fy, q), f4_at(xyl, q) - v, s);
    s = fmaf(h4_at(fyh, q), f4_at(xyh, q) - v, s);
    s = fmaf(h4_at(fz, q), f4_at(xzl, q) - v, s);
    s = fmaf(h4_at(fzh, q), f4_at(xzh, q) - v, s);
    if (dd16) s = fmaf(-dd_h(dd16, c0 + q), v, s);
    r[q] = f4_at(bb, q) - s * inv_fs;
  }
}

// residual + restriction with 16-byte fine rows (fine nx a multiple of 4): a
// thread owns coarse cells (2m, 2m + 1) of a coarse row, i.e. one 4-cell chunk
// of each of its four fine rows; children summed in k_resid_restrict_h's order
__global__ void k_resid_restrict_h4(const float *__restrict__ x, const float *__restrict__ b,
                                    const __half *__restrict__ hx, const __half *__restrict__ hy,
                                    const __half *__restrict__ hz, const __half *__restrict__ dd16,
                                    float inv_fs, Dims df, float *__restrict__ bc, Dims dc) {
  griddep_wait();
  const int m = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (m >= (df.nx >> 2) || J >= dc.ny) return;
  float s0 = 0.f, s1 = 0.f, r[4];
#pragma unroll
  for (int row = 0; row < 4; ++row) {  // (dj, dk) = (0,0), (1,0), (0,1), (1,1)
    resid_h4(x, b, hx, hy, hz, dd16, inv_fs, df, 4 * m, 2 * J + (row & 1), 2 * K + (row >> 1), r);
    s0 += r[0];
    s0 += r[1];
    s1 += r[2];
    s1 += r[3];
  }
  bc[at(dc, 2 * m, J, K)] = 0.5f * s0;
  bc[at(dc, 2 * m + 1, J, K)] = 0.5f * s1;
}

template <typename T>
__global__ void k_resid_restrict(const T *__restrict__ x, const T *__restrict__ b,
                                 const T *__restrict__ bx, const T *__restrict__ by,
                                 const T *__restrict__ bz, const T *__restrict__ diag, Dims df,
                                 T *__restrict__ bc, Dims dc) {
  griddep_wait();
  int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (I >= dc.nx || J >= dc.ny) return;
  resid_restrict_cell<T>(x, b, bx, by, bz, diag, df, bc, dc, I, J, K);
}

// ------------------------------------- A8: prolongation + correction
// piecewise-constant: each fine cell adds its parent's correction
template <typename T>
__global__ void k_prolong(T *__restrict__ x, const T *__restrict__ ec, Dims df, Dims dc) {
  griddep_wait();
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= df.nx || j >= df.ny) return;
  x[at(df, i, j, k)] += ec[at(dc, i >> 1, j >> 1, k >> 1)];
}

// The same with 16-byte accesses: a thread adds the corrections of its
// parents to 16/sizeof(T) consecutive cells of a row (nx a multiple of that;
// rows stay 16-byte aligned).  The scalar form is latency-bound at ~21% of HBM.
template <typename T>
__global__ void k_prolong_vec(T *__restrict__ x, const T *__restrict__ ec, Dims df, Dims dc) {
  griddep_wait();
  constexpr int W = 16 / sizeof(T);  // cells per thread (FP32: 4, FP64: 2)
  const int t = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (t >= df.nx / W || j >= df.ny) return;
  const int i = W * t;
  T *xr = x + at(df, i, j, k);
  const T *er = ec + at(dc, i >> 1, j >> 1, k >> 1);
  if (W == 4) {
    float4 v = *reinterpret_cast<float4 *>(xr);
    const float2 e = *reinterpret_cast<const float2 *>(er);
    v.x += e.x;
    v.y += e.x;
    v.z += e.y;
    v.w += e.y;
    *reinterpret_cast<float4 *>(xr) = v;
  } else {
    double2 v = *reinterpret_cast<double2 *>(xr);
    const double e = *reinterpret_cast<const double *>(er);
    v.x += e;
    v.y += e;
    *reinterpret_cast<double2 *>(xr) = v;
  }
}

// --------------------------------------------------------- Krylov kernels
// Scalars kept on the device between kernels (no host round trip).
enum { S_RZ = 0, S_RZOLD, S_DQ, S_ALPHA, S_BETA, S_RR, S_BB, S_MEAN, S_TMP, S_COUNT };
enum { OP_STORE = 0, OP_ALPHA, OP_BETA, OP_MEAN };

// Stencil kernels with a reduction walk a column of `zper` planes per
// thread (grid z = ceil(nz / zper)), so the partial-sum count stays ~2k.
// q = At d; per-block partial of d.q
template <typename T>
__global__ void k_apply_dot(const T *__restrict__ dv, T *__restrict__ q, const T *__restrict__ bx,
                            const T *__restrict__ by, const T *__restrict__ bz,
                            const T *__restrict__ diag, const T *__restrict__ dd, Dims d,
                            int zper, double *__restrict__ partial) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  int k0 = blockIdx.z * zper, k1 = min(d.nz, k0 + zper);
  T acc = 0;
  if (i < d.nx && j < d.ny)
    for (int k = k0; k < k1; ++k) {
      size_t c = at(d, i, j, k);
      T s = op_at(dv, bx, by, bz, diag, dd, d, i, j, k);
      q[c] = s;
      acc = fma(s, dv[c], acc);
    }
  double t = block_sum((double)acc);
  if (thread0()) partial[block_linear_id()] = t;
}

// q = At d (FP32 difference form, op_at's arithmetic per cell) and per-block
// partials of d.q, with 16-byte rows (nx a multiple of 4): a thread owns a
// 4-cell x-chunk in each of its zper planes and loads it as vectors.
// XPBY: the CG direction update d = z + beta d (k_xpby's operation, d = z on
// the first iteration) fused in: every value of d the stencil needs is formed
// from z and the old direction dv, and the thread's own chunk of the new
// direction is stored to dnew (a second buffer: other blocks still read dv).
__device__ __forceinline__ float4 xpby4(const float *__restrict__ z, const float *__restrict__ d,
                                        size_t c, float beta, int first) {
  const float4 zz = *reinterpret_cast<const float4 *>(z + c);
  if (first) return zz;
  const float4 dd = *reinterpret_cast<const float4 *>(d + c);
  return make_float4(fmaf(beta, dd.x, zz.x), fmaf(beta, dd.y, zz.y), fmaf(beta, dd.z, zz.z),
                     fmaf(beta, dd.w, zz.w));
}
template <bool XPBY>
__global__ void __launch_bounds__(BX * BY)
k_apply_dot4(const float *__restrict__ dv, float *__restrict__ q, const float *__restrict__ bx,
             const float *__restrict__ by, const float *__restrict__ bz,
             const float *__restrict__ dd32, Dims d, int zper, double *__restrict__ partial,
             const float *__restrict__ z, float *__restrict__ dnew,
             const double *__restrict__ scal, int first) {
  griddep_wait();
  const float beta = XPBY && !first ? (float)scal[S_BETA] : 0.f;
  auto ld4 = [&](size_t c) -> float4 {
    if (XPBY) return xpby4(z, dv, c, beta, first);
    return *reinterpret_cast<const float4 *>(dv + c);
  };
  auto ld1 = [&](size_t c) -> float {
    if (XPBY) return first ? z[c] : fmaf(beta, dv[c], z[c]);
    return dv[c];
  };
  const int t = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int k0 = blockIdx.z * zper, k1 = min(d.nz, k0 + zper);
  float acc = 0.f;
  if (t < (d.nx >> 2) && j < d.ny)
    for (int k = k0; k < k1; ++k) {
      const int i0 = 4 * t;
      const size_t c0 = at(d, i0, j, k);
      const size_t cyl = at(d, i0, wlo(j, d.ny), k), cyh = at(d, i0, whi(j, d.ny), k);
      const size_t czl = at(d, i0, j, wlo(k, d.nz)), czh = at(d, i0, j, whi(k, d.nz));
      const size_t ce = at(d, whi(i0 + 3, d.nx), j, k);
      const float4 xc = ld4(c0);
      const float4 xyl = ld4(cyl), xyh = ld4(cyh), xzl = ld4(czl), xzh = ld4(czh);
      if (XPBY) *reinterpret_cast<float4 *>(dnew + c0) = xc;
      const float4 fx = *reinterpret_cast<const float4 *>(bx + c0);
      const float4 fy = *reinterpret_cast<const float4 *>(by + c0);
      const float4 fyh = *reinterpret_cast<const float4 *>(by + cyh);
      const float4 fz = *reinterpret_cast<const float4 *>(bz + c0);
      const float4 fzh = *reinterpret_cast<const float4 *>(bz + czh);
      const float fxe = bx[ce], xp = ld1(ce), xm = ld1(at(d, wlo(i0, d.nx), j, k));
      float4 out;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float v = f4_at(xc, e);
        const float x_l = e > 0 ? f4_at(xc, e - 1) : xm, x_h = e < 3 ? f4_at(xc, e + 1) : xp;
        float s = f4_at(fx, e) * (x_l - v);
        s = fmaf(e < 3 ? f4_at(fx, e + 1) : fxe, x_h - v, s);
        s = fmaf(f4_at(fy, e), f4_at(xyl, e) - v, s);
        s = fmaf(f4_at(fyh, e), f4_at(xyh, e) - v, s);
        s = fmaf(f4_at(fz, e), f4_at(xzl, e) - v, s);
        s = fmaf(f4_at(fzh, e), f4_at(xzh, e) - v, s);
        if (dd32) s = fmaf(-dd32[c0 + e], v, s);
        if (e == 0) out.x = s; else if (e == 1) out.y = s; else if (e == 2) out.z = s; else out.w = s;
        acc = fmaf(s, v, acc);
      }
      *reinterpret_cast<float4 *>(q + c0) = out;
    }
  const double tot = block_sum((double)acc);
  if (thread0()) partial[block_linear_id()] = tot;
}

// r = b - At x (scaled), per-block partial of r.r; zero != 0: x = 0, r = b.
template <typename T>
__global__ void k_residual(const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ r,
                           const T *__restrict__ bx, const T *__restrict__ by,
                           const T *__restrict__ bz, const T *__restrict__ diag, Dims d, int zper,
                           double *__restrict__ partial, int zero) {
  const T *dd = nullptr;  // diag holds the outflow diagonal
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  int k0 = blockIdx.z * zper, k1 = min(d.nz, k0 + zper);
  double acc = 0.0;
  if (i < d.nx && j < d.ny)
    for (int k = k0; k < k1; ++k) {
      size_t c = at(d, i, j, k);
      T v = zero ? b[c] : resid_at(x, b, bx, by, bz, diag, dd, d, i, j, k);
      r[c] = v;
      acc = fma((double)v, (double)v, acc);
    }
  double t = block_sum(acc);
  if (thread0()) partial[block_linear_id()] = t;
}

// mixed precision outer residual: r64 = b - At64 x64 (FP64), r32 = fl32(r64)
__global__ void k_residual_mixed(const double *__restrict__ x, const double *__restrict__ b,
                                 float *__restrict__ r32, const double *__restrict__ bx,
                                 const double *__restrict__ by, const double *__restrict__ bz,
                                 const double *__restrict__ diag, Dims d, int zper,
                                 double *__restrict__ partial, int zero) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  int k0 = blockIdx.z * zper, k1 = min(d.nz, k0 + zper);
  double acc = 0.0;
  if (i < d.nx && j < d.ny)
    for (int k = k0; k < k1; ++k) {
      size_t c = at(d, i, j, k);
      double v = zero ? b[c] : resid_at(x, b, bx, by, bz, diag, (const double *)nullptr, d, i, j, k);
      r32[c] = (float)v;
      acc = fma(v, v, acc);
    }
  double t = block_sum(acc);
  if (thread0()) partial[block_linear_id()] = t;
}

// Grid-stride vector kernels: fixed grid (deterministic partial order).
// When every operand is 16-byte aligned (internal buffers always are; a
// caller's p usually is) they move 16 bytes per load (float4 / double2), two
// vectors per iteration, which keeps enough loads in flight to stream HBM.
constexpr int VEC_THREADS = 256;

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ static float at(const V &v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
  }
  __device__ static void set(V &v, int i, float a) {
    if (i == 0) v.x = a; else if (i == 1) v.y = a; else if (i == 2) v.z = a; else v.w = a;
  }
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ static double at(const V &v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static void set(V &v, int i, double a) {
    if (i == 0) v.x = a; else v.y = a;
  }
};
__device__ __forceinline__ bool aligned16(const void *a, const void *b = nullptr,
                                          const void *c = nullptr, const void *d = nullptr) {
  return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) & 15) == 0;
}

template <typename T>
__global__ void __launch_bounds__(VEC_THREADS, 4)
k_dot(const T *__restrict__ a, const T *__restrict__ b, size_t n, double *__restrict__ partial) {
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int W = VT::W;
  T acc = 0;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if (aligned16(a, b)) {
    const size_t nv = n / W;
    const V *av = reinterpret_cast<const V *>(a), *bv = reinterpret_cast<const V *>(b);
    for (size_t e = tid; e < nv; e += stride) {
      const V x = av[e], y = bv[e];
#pragma unroll
      for (int q = 0; q < W; ++q) acc = fma(VT::at(x, q), VT::at(y, q), acc);
    }
    done = nv * W;
  }
  for (size_t e = done + tid; e < n; e += stride) acc = fma(a[e], b[e], acc);
  double t = block_sum((double)acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// x += alpha d; r -= alpha q; partial r.r
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS, 4)
k_axpy2(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ dv,
                        const T *__restrict__ q, size_t n, const double *__restrict__ scal,
                        double *__restrict__ partial) {
  griddep_wait();
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int W = VT::W;
  const T alpha = (T)scal[S_ALPHA];
  T acc = 0;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if (aligned16(x, r, dv, q)) {
    const size_t nv = n / W;
    V *xv = reinterpret_cast<V *>(x), *rv = reinterpret_cast<V *>(r);
    const V *dvv = reinterpret_cast<const V *>(dv), *qv = reinterpret_cast<const V *>(q);
    for (size_t e = tid; e < nv; e += stride) {
      V xe = xv[e], re = rv[e];
      const V de = dvv[e], qe = qv[e];
#pragma unroll
      for (int k = 0; k < W; ++k) {
        VT::set(xe, k, fma(alpha, VT::at(de, k), VT::at(xe, k)));
        const T rk = fma(-alpha, VT::at(qe, k), VT::at(re, k));
        VT::set(re, k, rk);
        acc = fma(rk, rk, acc);
      }
      xv[e] = xe;
      rv[e] = re;
    }
    done = nv * W;
  }
  for (size_t e = done + tid; e < n; e += stride) {
    x[e] = fma(alpha, dv[e], x[e]);
    T rv = fma(-alpha, q[e], r[e]);
    r[e] = rv;
    acc = fma(rv, rv, acc);
  }
  double t = block_sum((double)acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// d = z + beta d (first iteration: d = z)
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS, 4)
k_xpby(T *__restrict__ dv, const T *__restrict__ z, size_t n,
                       const double *__restrict__ scal, int first) {
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int W = VT::W;
  const T beta = first ? (T)0 : (T)scal[S_BETA];
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if (aligned16(dv, z)) {
    const size_t nv = n / W;
    V *dvv = reinterpret_cast<V *>(dv);
    const V *zv = reinterpret_cast<const V *>(z);
    for (size_t e = tid; e < nv; e += stride) {
      const V ze = zv[e];
      V de = first ? ze : dvv[e];
      if (!first) {
#pragma unroll
        for (int k = 0; k < W; ++k) VT::set(de, k, fma(beta, VT::at(de, k), VT::at(ze, k)));
      }
      dvv[e] = de;
    }
    done = nv * W;
  }
  for (size_t e = done + tid; e < n; e += stride) dv[e] = first ? z[e] : fma(beta, dv[e], z[e]);
}

// x += y (stationary iteration update)
template <typename T>
__global__ void k_add(T *__restrict__ x, const T *__restrict__ y, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    x[e] += y[e];
}

// x64 += e32, then e32 = 0 (accumulation of an FP32 correction in FP64)
// x += (double) e, e = 0: four cells per step (16-byte e, two 16-byte x
// accesses) when both arrays start 16-byte aligned (x may be a caller's
// view), then the tail
__global__ void k_add_f32(double *__restrict__ x, float *__restrict__ e, size_t n) {
  const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(e)) & 15) == 0;
  const size_t n4 = vec ? n / 4 : 0, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += stride) {
    float4 *ep = reinterpret_cast<float4 *>(e) + q;
    double2 *xp = reinterpret_cast<double2 *>(x) + 2 * q;
    const float4 v = *ep;
    double2 a = xp[0], c = xp[1];
    a.x += (double)v.x;
    a.y += (double)v.y;
    c.x += (double)v.z;
    c.y += (double)v.w;
    xp[0] = a;
    xp[1] = c;
    *ep = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (size_t k = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    x[k] += (double)e[k];
    e[k] = 0.f;
  }
}

// y = (double) x
__global__ void k_f32_to_f64(const float *__restrict__ x, double *__restrict__ y, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    y[k] = (double)x[k];
}

// g = fl32(a u + b v)
__global__ void k_lincomb_f32(float *__restrict__ g, double a, const double *__restrict__ u,
                              double b, const double *__restrict__ v, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    g[k] = (float)fma(a, u[k], b * v[k]);
}

// dst32 = fl32(src64), per-block partial of src.src (FP64)
__global__ void k_to_f32_norm(const double *__restrict__ src, float *__restrict__ dst, size_t n,
                              double *__restrict__ partial) {
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const double v = src[e];
    dst[e] = (float)v;
    acc = fma(v, v, acc);
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

template <typename T>
__global__ void k_sum(const T *__restrict__ a, size_t n, double *__restrict__ partial) {
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    acc += (double)a[e];
  double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// x -= mean (scal[S_MEAN]); optional partial of the new x.x
__global__ void k_sub_mean(double *__restrict__ x, size_t n, const double *__restrict__ scal,
                           double *__restrict__ partial) {
  double m = scal[S_MEAN];
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double v = x[e] - m;
    x[e] = v;
    acc = fma(v, v, acc);
  }
  double t = block_sum(acc);
  if (partial != nullptr && threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Single-block final reduction of the partials in a fixed order, then an
// operation on the device scalars.
__global__ void k_reduce(const double *__restrict__ partial, int np, double *__restrict__ scal,
                         int op, int slot, double count) {
  griddep_wait();
  double acc = 0.0;
  for (int e = threadIdx.x; e < np; e += blockDim.x) acc += partial[e];
  double s = block_sum(acc);
  if (threadIdx.x == 0) {
    switch (op) {
      case OP_STORE: scal[slot] = s; break;
      case OP_ALPHA: scal[S_DQ] = s; scal[S_ALPHA] = scal[S_RZ] / s; break;
      case OP_BETA:
        scal[S_RZOLD] = scal[S_RZ];
        scal[S_RZ] = s;
        scal[S_BETA] = s / scal[S_RZOLD];
        break;
      case OP_MEAN: scal[S_MEAN] = s / count; break;
    }
  }
}

// --------------------------------------------------------- assembly (A3)
// bt = h^2 rhs + Jt; per-block partial sum (for the mean)
__global__ void k_assemble(const double *__restrict__ rhs, const double *__restrict__ Jt,
                           double *__restrict__ b, size_t n, double h2,
                           double *__restrict__ partial) {
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double v = fma(h2, rhs[e], Jt[e]);
    b[e] = v;
    acc += v;
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// bt = h^2 div_h u* + Jt = h * sum(u_high - u_low) + Jt, fused divergence
__global__ void k_assemble_u(const double *__restrict__ ux, const double *__restrict__ uy,
                             const double *__restrict__ uz, const double *__restrict__ Jt,
                             double *__restrict__ b, Dims d, int zper, int kb0, double h,
                             double *__restrict__ partial) {
  // kb0: z-block offset of this launch (a slab of the z-blocks); partial is
  // indexed by the global block
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  int k0 = (blockIdx.z + kb0) * zper, k1 = min(d.nz, k0 + zper);
  double acc = 0.0;
  if (i < d.nx && j < d.ny)
    for (int k = k0; k < k1; ++k) {
      size_t c = at(d, i, j, k);
      double s = ux[at(d, whi(i, d.nx), j, k)] - ux[c] + uy[at(d, i, whi(j, d.ny), k)] - uy[c] +
                 uz[at(d, i, j, whi(k, d.nz))] - uz[c];
      double v = fma(h, s, Jt[c]);
      b[c] = v;
      acc += v;
    }
  double t = block_sum(acc);
  if (thread0()) partial[block_linear_id() + (size_t)kb0 * gridDim.x * gridDim.y] = t;
}

// div_h u = sum over axes of (u_high - u_low) / h
__global__ void k_divergence(const double *__restrict__ ux, const double *__restrict__ uy,
                             const double *__restrict__ uz, double *__restrict__ dv, Dims d,
                             double h) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  size_t c = at(d, i, j, k);
  double s = ux[at(d, whi(i, d.nx), j, k)] - ux[c] + uy[at(d, i, whi(j, d.ny), k)] - uy[c] +
             uz[at(d, i, j, whi(k, d.nz))] - uz[c];
  dv[c] = s / h;
}

// ------------------------------------------------- A15: velocity correction
// u_f -= beta_f (p_b - p_a - [p]_{a->b}) / h on the three low faces of each
// cell; wall faces have beta = 0 and keep u*.  Planes k0 .. k0 + gridDim.z - 1.
// With a mass flux (mdot not null) an interface face stores its liquid-side
// velocity: the flux-jump share of the liquid row is removed from the
// correction (+share B when the low cell is liquid, -share B when the high
// cell is).
__global__ void k_project(const double *__restrict__ p, const double *__restrict__ phi,
                          const double *__restrict__ kap, const double *__restrict__ bx,
                          const double *__restrict__ by, const double *__restrict__ bz,
                          double *__restrict__ ux, double *__restrict__ uy,
                          double *__restrict__ uz, Dims d, int k0, double sig, double ih,
                          const double *__restrict__ mdot, double rl, double rg) {
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z + k0;
  if (i >= d.nx || j >= d.ny) return;
  size_t c = at(d, i, j, k);
  double pc = p[c], fc = phi[c], kc = kap[c];
  size_t xl = at(d, wlo(i, d.nx), j, k), yl = at(d, i, wlo(j, d.ny), k),
         zl = at(d, i, j, wlo(k, d.nz));
  const bool g = gas(fc);
  double dx = pc - p[xl], dy = pc - p[yl], dz = pc - p[zl];
  if (gas(phi[xl]) != g) dx -= gfm_jump(phi[xl], fc, kap[xl], kc, sig);
  if (gas(phi[yl]) != g) dy -= gfm_jump(phi[yl], fc, kap[yl], kc, sig);
  if (gas(phi[zl]) != g) dz -= gfm_jump(phi[zl], fc, kap[zl], kc, sig);
  double vx = fma(-bx[c] * ih, dx, ux[c]);
  double vy = fma(-by[c] * ih, dy, uy[c]);
  double vz = fma(-bz[c] * ih, dz, uz[c]);
  if (mdot) {
    const double jinv = 1.0 / rg - 1.0 / rl, mc = mdot[c];
    const size_t nb[3] = {xl, yl, zl};
    const double bf[3] = {bx[c], by[c], bz[c]};
    double *v[3] = {&vx, &vy, &vz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double pa = phi[nb[q]];
      if (gas(pa) == g || bf[q] == 0.0) continue;
      const double B = flux_jump_B(pa, fc, mdot[nb[q]], mc, jinv);
      if (!gas(pa))  // low cell liquid: its side's flux
        *v[q] += flux_share(pa, fc, bf[q], rl, rg) * B;
      else           // high cell (this one) liquid
        *v[q] -= flux_share(fc, pa, bf[q], rl, rg) * B;
    }
  }
  ux[c] = vx;
  uy[c] = vy;
  uz[c] = vz;
}

// ------------------------------------------------ outflow boundary planes
// Finest level: the coefficient of every outflow boundary face, 1/rho of the
// fluid of the cell next to it (its ghost lies in that fluid).  side: 0..5
// (x low, x high, y low, y high, z low, z high); the plane layout as in
// BndPlanes.
__global__ void k_bnd_init(const double *__restrict__ phi, double *__restrict__ plane, Dims d,
                           int side, double irl, double irg) {
  const int axis = side >> 1, hi = side & 1;
  const int na = axis == 0 ? d.ny : d.nx, nb = axis == 2 ? d.ny : d.nz;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= na * nb) return;
  const int u = e % na, v = e / na;
  int i, j, k;
  if (axis == 0) { i = hi ? d.nx - 1 : 0; j = u; k = v; }
  else if (axis == 1) { j = hi ? d.ny - 1 : 0; i = u; k = v; }
  else { k = hi ? d.nz - 1 : 0; i = u; j = v; }
  plane[e] = gas(phi[at(d, i, j, k)]) ? irg : irl;
}

// A coarse boundary face is the mean of the four fine faces that tile it.
__global__ void k_bnd_coarsen(const double *__restrict__ fine, double *__restrict__ coarse,
                              int na, int nb) {  // coarse plane na x nb, fine 2na x 2nb
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= na * nb) return;
  const int u = e % na, v = e / na, fa = 2 * na;
  coarse[e] = 0.25 * (fine[2 * u + fa * 2 * v] + fine[2 * u + 1 + fa * 2 * v] +
                      fine[2 * u + fa * (2 * v + 1)] + fine[2 * u + 1 + fa * (2 * v + 1)]);
}

// y = scale * v (used to unscale J and the operator for the test API)
// y = scale v; y may be v (in place), so the pointers are not restrict
__global__ void k_scale(const double *v, double *y, size_t n, double scale) {
  // two cells per step when both arrays start 16-byte aligned, then the tail
  const bool vec = ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  const size_t n2 = vec ? n / 2 : 0, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n2; q += stride) {
    const double2 a = reinterpret_cast<const double2 *>(v)[q];
    reinterpret_cast<double2 *>(y)[q] = make_double2(a.x * scale, a.y * scale);
  }
  for (size_t e = 2 * n2 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride)
    y[e] = v[e] * scale;
}

}  // namespace mp
