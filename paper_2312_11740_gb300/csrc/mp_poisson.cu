// Host driver and C-ABI of the pressure-Poisson hot path (see include/mp_poisson.h).
//
// Solver: conjugate gradients on the h^2-scaled system At x = bt,
// preconditioned by one symmetric geometric-multigrid V-cycle (red-black
// Gauss-Seidel: red then black before the coarse correction, black then red
// after; mean restriction; piecewise-constant prolongation; face-averaged
// coarse coefficients; dense FP64 inverse on the coarsest level).  Mixed
// precision wraps an FP32 inner solve in FP64 iterative refinement: the
// outer residual, the solution accumulation and the coarsest solve are FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mp_net.h"
#include "../../include/mp_poisson.h"
#include "mp_kernels.cuh"
#include "mp_sweep.cuh"
#include "mp_ctail.cuh"
#include "mp_deflate.cuh"

using namespace mp;

namespace {

constexpr int MAX_COARSE = 512;
constexpr int VEC_BLOCKS = 152 * 4;  // fixed grid for vector kernels: 4 resident per SM (152 SMs)

struct Level {
  Dims d;
  size_t n = 0;
  int nu1 = 2, nu2 = 2;
  double *bx = nullptr, *by = nullptr, *bz = nullptr, *diag = nullptr, *idiag = nullptr;
  float *bx32 = nullptr, *by32 = nullptr, *bz32 = nullptr, *idiag32 = nullptr;
  __half *bx16 = nullptr, *by16 = nullptr, *bz16 = nullptr;  // FP32 V-cycle faces, x fs16
  double *b = nullptr, *e = nullptr;   // coarse-level rhs / correction (levels >= 1)
  float *b32 = nullptr, *e32 = nullptr;
  float *t32 = nullptr;  // second FP32 iterate of the fused sweep (levels it runs on)
  int ftx = 0, fty = 0, fchunk = 0;  // fused sweep grid: tiles in x, y; z-chunks
  // outflow sides: the boundary-face coefficients per side (planes, null for
  // other sides) and the per-cell outflow diagonal (null without outflow)
  double *bnd[6] = {};
  double *dd = nullptr;
  float *dd32 = nullptr;
  __half *dd16 = nullptr;
};

enum KernelId {
  K_CURV, K_FACES, K_JUMP, K_DIAG, K_COARSEN, K_DENSE, K_GJ,
  K_RBGS64, K_RBGS32, K_RBGS32F, K_TAIL64, K_TAIL32, K_CTAIL32, K_RESTR64, K_RESTR32, K_PROL64, K_PROL32, K_COARSE64, K_COARSE32,
  K_APPLY64, K_APPLY32, K_RESID64, K_RESID32, K_RESIDMIX, K_DOT64, K_DOT32, K_AXPY64, K_AXPY32,
  K_XPBY64, K_XPBY32, K_ADD64, K_ADD32, K_ADDF32, K_SUM, K_SUBMEAN, K_REDUCE, K_ASSEMBLE,
  K_ASSEMBLE_U, K_PROJECT, K_DIV, K_SCALE, K_DEFL, K_DEFL_LABEL, K_DEFL_DOT, K_COUNT
};
const char *const kKernelNames[K_COUNT] = {
  "curvature", "gfm_faces", "jump", "diag", "coarsen_faces", "dense_build", "gauss_jordan",
  "rbgs_f64", "rbgs_f32", "rbgs_f32_fused", "coarse_tail_f64", "coarse_tail_f32",
  "coarse_cluster_f32",
  "resid_restrict_f64", "resid_restrict_f32", "prolong_f64",
  "prolong_f32", "coarse_solve_f64", "coarse_solve_f32io", "apply_dot_f64", "apply_dot_f32",
  "residual_f64", "residual_f32", "residual_mixed", "dot_f64", "dot_f32", "axpy2_f64",
  "axpy2_f32", "xpby_f64", "xpby_f32", "add_f64", "add_f32", "add_f32_to_f64", "sum",
  "sub_mean", "reduce", "assemble", "assemble_u", "project", "divergence", "scale",
  "deflation_band", "deflation_label", "deflation_dot"};
constexpr int MAX_LEVELS = 16;
constexpr int TAIL32_NU_MAX = 4;  // sweeps per level in the one-CTA FP32 tail
constexpr size_t CT_SMEM_MAX = 200 * 1024;  // shared memory per CTA of the cluster tail
constexpr int EVENT_POOL = 4096;
constexpr int MAX_SLABS = 8;  // z-slabs of the host-buffer step's copy pipeline

struct ProfEntry {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0;
};
struct Pending {
  int id, level;
  cudaEvent_t a, b;
  double bytes;
};

}  // namespace

struct mp_poisson {
  mp_grid g{};
  int per = 0;
  int outflow = 0;  // bits 2a (low) and 2a+1 (high): outflow (p = 0) sides of axis a
  double h = 1.0, rho_l = 1.0, rho_g = 1.0, sigma = 0.0;
  mp_opts opts{};
  cudaStream_t st = nullptr;
  std::vector<Level> L;
  size_t n = 0;
  // fine-level FP64 fields
  double *phi = nullptr, *kap = nullptr, *Jt = nullptr, *b = nullptr;
  double *mdot = nullptr;  // phase-change mass flux per cell (mp_poisson_set_mass_flux)
  int has_mdot = 0;
  double *r = nullptr, *z = nullptr, *dv = nullptr, *q = nullptr;
  // fine-level FP32 inner-solve vectors
  float *r32 = nullptr, *e32 = nullptr, *z32 = nullptr, *d32 = nullptr, *q32 = nullptr;
  float *d32b = nullptr;  // second direction buffer (fused direction update + operator)
  // host-buffer step staging
  double *ux = nullptr, *uy = nullptr, *uz = nullptr, *pst = nullptr;
  // coarsest level
  double *Maug = nullptr, *Minv = nullptr;
  int nc = 0;
  // reductions
  double *partial = nullptr, *scal = nullptr, *scal_h = nullptr;
  int npart = 0;
  double bnorm = 0.0;
  mp_stats stats{};
  // deflation by the gas components (mp_deflate.cuh)
  int *lab = nullptr, *comp = nullptr, *band = nullptr, *cnt = nullptr, *dint = nullptr;
  int *roots = nullptr;
  int *troots = nullptr;  // tile roots of the labelling (up to tcap)
  int tcap = 0;
  unsigned char *bflag = nullptr;  // band flag per cell (compaction)
  int defl_m = 0, defl_nband = 0;
  double beta_max = 1.0, ztb_scale = 1.0;
  float fs16 = 1.f;  // scale of the FP16 faces (a power of two)
  int diag_mode = 0;  // per-level arrays formed by k_diag for this geometry (bits: 1 FP64, 2 FP32)
  double *einv = nullptr, *coef = nullptr, *dscale = nullptr;
  float *coef32 = nullptr;
  unsigned long long *acc_a = nullptr, *acc_b = nullptr, *acc_ztb = nullptr, *dmax = nullptr;
  int *hint = nullptr;  // pinned host copy of dint
  mp_net_handle net = nullptr;  // learned initial guess (initial_guess = 2)
  int net_factor = 1;           // solver grid / network grid (1 or 2)
  std::vector<void *> allocs;
  // launch accounting / CUDA-event profiling
  ProfEntry prof[K_COUNT][MAX_LEVELS];
  int prof_on = 0;
  std::vector<cudaEvent_t> events;
  size_t ev_next = 0;
  std::vector<Pending> pending;
  // CUDA graphs of whole V-cycles, keyed by (type, rhs, x); launched on st
  struct Graph {
    int type;
    const void *rhs, *x;
    cudaGraphExec_t exec;
    std::vector<int> ids, levels;  // kernels in the graph, for launch accounting
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;  // private stream used only for capture
  // host-buffer step: copy stream and the events that order its z-slab copies
  // against the assembly and the velocity correction on st
  cudaStream_t cs = nullptr;
  cudaEvent_t xev[2 * MAX_SLABS + 2] = {};
  // first level of the one-CTA coarse tail per precision, and its smem bytes
  int tail64 = 0, tail32 = 0;
  // FP32 cluster tail (mp_ctail.cuh): its top level (-1: not used), shared memory per
  // CTA and the offset of its coarsest-rhs scratch
  int ctail32 = -1, ctail_scratch = 0;
  size_t ctail_bytes = 0;
  size_t tail64_bytes = 0, tail32_bytes = 0;
  bool capturing = false;
  std::vector<int> cap_ids, cap_levels;
};

namespace {

#define CK(call)                                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return MP_ERR_CUDA;      \
  } while (0)
#define CKS(call)                       \
  do {                                  \
    mp_status s_ = (call);              \
    if (s_ != MP_OK) return s_;         \
  } while (0)

dim3 cell_grid(const Dims &d) { return dim3((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, d.nz); }
dim3 half_grid(const Dims &d) {
  return dim3(((d.nx >> 1) + BX - 1) / BX, (d.ny + BY - 1) / BY, d.nz);
}
int cell_blocks(const Dims &d) {
  dim3 g = cell_grid(d);
  return (int)(g.x * g.y * g.z);
}
const dim3 kBlock(BX, BY, 1);

// Stencil+reduction kernels: each thread walks zper planes; about 2k blocks
// (measured: 16k blocks of 4 planes made k_apply_dot 40% slower).
int zper_of(const Dims &d) {
  long plane_blocks = (long)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY);
  long want = std::max<long>(1, 2048 / std::max<long>(1, plane_blocks));
  long zb = std::min<long>(d.nz, want);
  return (int)((d.nz + zb - 1) / zb);
}
dim3 zgrid(const Dims &d) {
  int zp = zper_of(d);
  return dim3((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, (d.nz + zp - 1) / zp);
}
// the same decomposition for kernels that own 4-cell x-chunks (nx % 4 == 0)
Dims chunk_dims(const Dims &d) {
  Dims q = d;
  q.nx = d.nx / 4;
  return q;
}
int zblocks(const Dims &d) {
  dim3 g = zgrid(d);
  return (int)(g.x * g.y * g.z);
}
// dynamic shared memory of the one-CTA coarse tail: FP32 levels up to ~16^3;
// FP64 only the smallest levels (one SM's FP64 rate is the limit there)
constexpr size_t TAIL_BUDGET32 = 200 * 1024, TAIL_BUDGET64 = 48 * 1024;

template <typename T>
mp_status dalloc(mp_poisson *hd, T **p, size_t count) {
  void *v = nullptr;
  if (cudaMalloc(&v, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return MP_ERR_OOM;
  }
  hd->allocs.push_back(v);
  // every buffer starts finite (a stencil multiplies wall neighbours by a 0 face)
  if (cudaMemset(v, 0, count * sizeof(T) + 16) != cudaSuccess) return MP_ERR_CUDA;
  *p = (T *)v;
  return MP_OK;
}

mp_status launch_ok() { return cudaGetLastError() == cudaSuccess ? MP_OK : MP_ERR_CUDA; }

// Resolve recorded event pairs into per-kernel times (stream must be idle).
void prof_resolve(mp_poisson *hd) {
  for (const Pending &p : hd->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      hd->prof[p.id][p.level].ms += ms;
      hd->prof[p.id][p.level].bytes += p.bytes;
    }
  }
  hd->pending.clear();
  hd->ev_next = 0;
}

void prof_begin(mp_poisson *hd, int id, int level) {
  if (hd->capturing) {
    hd->cap_ids.push_back(id);
    hd->cap_levels.push_back(level);
    return;
  }
  hd->prof[id][level].launches++;
  if (!hd->prof_on) return;
  if (hd->ev_next + 2 > hd->events.size()) {
    cudaStreamSynchronize(hd->st);
    prof_resolve(hd);
  }
  cudaEventRecord(hd->events[hd->ev_next], hd->st);
}

void prof_end(mp_poisson *hd, int id, int level, double bytes) {
  if (!hd->prof_on || hd->capturing) return;
  cudaEvent_t a = hd->events[hd->ev_next], b = hd->events[hd->ev_next + 1];
  cudaEventRecord(b, hd->st);
  hd->ev_next += 2;
  hd->pending.push_back(Pending{id, level, a, b, bytes});
}

// Launch on the handle's stream, counted per (kernel, level) and, when
// profiling is on, bracketed by CUDA events.  BYTES is the algorithmic
// traffic of the launch (unique bytes it must read and write).
#define LAUNCH(hd, id, level, bytes, kern, grid, block, ...)      \
  do {                                                            \
    prof_begin((hd), (id), (level));                              \
    kern<<<(grid), (block), 0, (hd)->st>>>(__VA_ARGS__);          \
    prof_end((hd), (id), (level), (double)(bytes));               \
  } while (0)
// Launch with programmatic stream serialization: the kernel's blocks may be
// scheduled while the previous kernel on the stream finishes (hiding the
// launch gap of the small coarse-level kernels); the kernel must begin with
// griddep_wait().  Falls back to an ordinary launch if the attribute is refused.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...) != cudaSuccess) {
    cudaGetLastError();
    kern<<<grid, block, smem, st>>>(static_cast<KArgs>(args)...);
  }
}
// LAUNCH for the V-cycle kernels (eager and profiled: an ordinary launch)
#define LAUNCH_PDL(hd, id, level, bytes, kern, grid, block, smem, ...)       \
  do {                                                                      \
    prof_begin((hd), (id), (level));                                        \
    if ((hd)->prof_on)                                                      \
      kern<<<(grid), (block), (smem), (hd)->st>>>(__VA_ARGS__);             \
    else                                                                    \
      launch_pdl(kern, (grid), (block), (smem), (hd)->st, __VA_ARGS__);     \
    prof_end((hd), (id), (level), (double)(bytes));                         \
  } while (0)
// the same with dynamic shared memory
#define LAUNCH_SMEM(hd, id, level, bytes, kern, grid, block, smem, ...) \
  do {                                                                  \
    prof_begin((hd), (id), (level));                                    \
    kern<<<(grid), (block), (smem), (hd)->st>>>(__VA_ARGS__);           \
    prof_end((hd), (id), (level), (double)(bytes));                     \
  } while (0)

template <typename T>
constexpr int kid(int id64, int id32) {
  return sizeof(T) == 8 ? id64 : id32;
}

// ---- reductions
// the phase-change mass flux the kernels read (null when none is set)
const double *mdot_of(const mp_poisson *hd) { return hd->has_mdot ? hd->mdot : nullptr; }

mp_status reduce(mp_poisson *hd, int np, int op, int slot, double count = 0.0) {
  LAUNCH(hd, K_REDUCE, 0, np * 8.0, k_reduce, 1, 1024, hd->partial, np, hd->scal, op, slot, count);
  return launch_ok();
}
// the same for a reduction whose predecessor on the stream is the kernel that
// wrote the partials: launched with programmatic serialization (k_reduce waits
// for that kernel before reading)
mp_status reduce_after(mp_poisson *hd, int np, int op, int slot) {
  LAUNCH_PDL(hd, K_REDUCE, 0, np * 8.0, k_reduce, 1, 1024, 0, (const double *)hd->partial, np,
             hd->scal, op, slot, 0.0);
  return launch_ok();
}

mp_status read_scalars(mp_poisson *hd) {
  CK(cudaMemcpyAsync(hd->scal_h, hd->scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                     hd->st));
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

// ---- per-precision level accessors
template <typename T> struct LV;
template <> struct LV<double> {
  static double *bx(Level &l) { return l.bx; }
  static double *by(Level &l) { return l.by; }
  static double *bz(Level &l) { return l.bz; }
  static double *diag(Level &l) { return l.diag; }
  static double *idiag(Level &l) { return l.idiag; }
  static double *b(Level &l) { return l.b; }
  static double *e(Level &l) { return l.e; }
  static double *dd(Level &l) { return l.dd; }
};
template <> struct LV<float> {
  static float *bx(Level &l) { return l.bx32; }
  static float *by(Level &l) { return l.by32; }
  static float *bz(Level &l) { return l.bz32; }
  static float *diag(Level &) { return nullptr; }  // FP32 operators use the difference form
  static float *idiag(Level &l) { return l.idiag32; }
  static float *b(Level &l) { return l.b32; }
  static float *e(Level &l) { return l.e32; }
  static float *dd(Level &l) { return l.dd32; }
};

// The FP32 cluster tail from level l down (one launch of a CT_CTAS cluster).
mp_status ctail_launch(mp_poisson *hd, int l, const float *rhs, float *x) {
  CtArgs a{};
  a.nlev = (int)hd->L.size() - l;
  a.Minv = hd->Minv;
  a.singular = hd->outflow == 0;
  int off = 0;
  double bytes = 0.0;
  for (int q = 0; q < a.nlev; ++q) {
    Level &t = hd->L[l + q];
    // the levels the one-CTA tail would take keep its sweep cap
    const int cap = l + q >= hd->tail32 ? TAIL32_NU_MAX : 1 << 20;
    const int ppc = std::max(1, t.d.nz / CT_CTAS);
    a.lv[q] = CtLevel{t.d, (int)t.n, std::min(t.nu1, cap), std::min(t.nu2, cap), ppc, off,
                      t.bx32, t.by32, t.bz32, t.idiag32, hd->outflow ? t.dd32 : nullptr};
    off += ct_slab_floats(t.d, ppc, hd->outflow != 0);
    bytes += 16.0 * t.n;
  }
  prof_begin(hd, K_CTAIL32, l);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CT_CTAS);
  cfg.blockDim = dim3(CTL_THREADS);
  cfg.dynamicSmemBytes = hd->ctail_bytes;
  cfg.stream = hd->st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CT_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = hd->prof_on ? 1 : 2;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_ctail, a, hd->ctail_scratch, rhs, x);
  if (e != cudaSuccess && cfg.numAttrs == 2) {  // without the programmatic launch
    cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_ctail, a, hd->ctail_scratch, rhs, x);
  }
  prof_end(hd, K_CTAIL32, l, bytes);
  if (e != cudaSuccess) return MP_ERR_CUDA;
  return launch_ok();
}

// One symmetric V-cycle with zero initial guess: x ~= At^-1 rhs on level l.
// Pre-smoothing sweeps red then black, post-smoothing black then red (the
// adjoint), so the cycle is a symmetric preconditioner.  Each colour is one
// in-place launch (a colour reads only the other colour).  The levels at
// the bottom run inside one CTA (k_tail).
template <typename T>
mp_status vcycle(mp_poisson *hd, int l, const T *rhs, T *x) {
  Level &lv = hd->L[l];
  if constexpr (sizeof(T) == 4) {
    if (l == hd->ctail32 && hd->opts.coarse_cluster) return ctail_launch(hd, l, rhs, x);
  }
  const int tail = sizeof(T) == 8 ? hd->tail64 : hd->tail32;
  if (l == tail && l < (int)hd->L.size() - 1) {
    TailArgs a{};
    a.nlev = (int)hd->L.size() - l;
    a.Minv = hd->Minv;
    a.singular = hd->outflow == 0;
    double bytes = 0.0;
    int off = 0;
    // the FP32 tail (levels <= 16^3, latency-bound at about a microsecond per
    // half-sweep) caps its sweeps at TAIL32_NU_MAX: measured, the deflated mixed
    // solve needs no more there (FP64 keeps the level's sweeps; the same cap
    // cost it iterations)
    const int cap = sizeof(T) == 4 ? TAIL32_NU_MAX : 1 << 20;
    for (int q = 0; q < a.nlev; ++q) {
      Level &t = hd->L[l + q];
      a.lv[q] = TailLevel{t.d, (int)t.n, std::min(t.nu1, cap), std::min(t.nu2, cap), off,
                          LV<T>::bx(t), LV<T>::by(t), LV<T>::bz(t), LV<T>::idiag(t),
                          LV<T>::dd(t)};
      off += (hd->outflow ? 7 : 6) * (int)t.n;
      bytes += 4.0 * t.n * sizeof(T);
    }
    size_t smem = sizeof(T) == 8 ? hd->tail64_bytes : hd->tail32_bytes;
    auto ktail = k_tail<T>;
    LAUNCH_PDL(hd, kid<T>(K_TAIL64, K_TAIL32), l, bytes, ktail, 1, TAIL_THREADS, smem, a, rhs, x);
    return launch_ok();
  }
  if (l == (int)hd->L.size() - 1) {
    LAUNCH_PDL(hd, kid<T>(K_COARSE64, K_COARSE32), l, lv.n * (lv.n * 8.0 + 2.0 * sizeof(T)),
               k_coarse_solve<T>, 1, 512, 0, hd->Minv, rhs, x, (int)lv.n, hd->outflow == 0 ? 1 : 0);
    return launch_ok();
  }
  Level &lc = hd->L[l + 1];
  T *bx = LV<T>::bx(lv), *by = LV<T>::by(lv), *bz = LV<T>::bz(lv);
  T *diag = LV<T>::diag(lv), *idiag = LV<T>::idiag(lv);
  const double sz = sizeof(T), nl = (double)lv.n;
  {
    dim3 hg = half_grid(lv.d);
    const int krb = kid<T>(K_RBGS64, K_RBGS32);
    // FP64 reads the stored 1/diag (FP64 division is costly on this part);
    // FP32 sweeps read FP16 faces and form 1/diag from them
    const double per = sizeof(T) == 8 ? 5.0 : 3.0;
    auto sweep = [&](int colour, int zero) -> mp_status {
      const double bytes = (zero ? per - 0.5 : per) * nl * sz;
      if constexpr (sizeof(T) == 4) {
        if (lv.d.nx % 4 == 0)  // 16-byte rows (level buffers are 256-byte aligned)
          LAUNCH_PDL(hd, krb, l, bytes, k_rbgs_h4,
                     dim3((lv.d.nx / 4 + BX - 1) / BX, (lv.d.ny + BY - 1) / BY, lv.d.nz), kBlock,
                     0, x, rhs, lv.bx16, lv.by16, lv.bz16, (const __half *)lv.dd16, lv.d, colour, zero,
                     hd->fs16);
        else
          LAUNCH_PDL(hd, krb, l, bytes, k_rbgs_h, hg, kBlock, 0, x, rhs, lv.bx16, lv.by16,
                     lv.bz16, (const __half *)lv.dd16, lv.d, colour, zero, hd->fs16);
      }
      else
        LAUNCH_PDL(hd, krb, l, bytes, k_rbgs<T>, hg, kBlock, 0, x, rhs, bx, by, bz, idiag, lv.d,
                   colour, zero);
      return MP_OK;
    };
    // FP32 levels with a fused-sweep grid: one launch per sweep, ping-pong
    // between x and t32 (pairs of sweeps end in x); an odd last sweep, and
    // every sweep of the other levels, is one in-place launch per colour
    const bool fused = sizeof(T) == 4 && hd->opts.smoother == 1 && lv.fchunk > 0 && !hd->outflow;
    auto fsweep = [&](const float *xin, float *xout, int c0, int zero) -> mp_status {
      FusedArgs fa{xin, xout, (const float *)rhs, lv.bx16, lv.by16, lv.bz16, lv.d, c0, zero,
                   hd->fs16, lv.ftx, lv.fty, lv.fchunk};
      // x, b and three face arrays read, x written (x not read by a first sweep)
      const double bytes = (zero ? 20.0 : 24.0) * nl;
      if (zero)
        LAUNCH_PDL(hd, K_RBGS32F, l, bytes, k_rbgs_fused<true>, lv.ftx * lv.fty * lv.fchunk,
                   FS_THREADS, FS_SMEM, fa);
      else
        LAUNCH_PDL(hd, K_RBGS32F, l, bytes, k_rbgs_fused<false>, lv.ftx * lv.fty * lv.fchunk,
                   FS_THREADS, FS_SMEM, fa);
      return MP_OK;
    };
    auto smooth = [&](int nu, int c0, int first_zero) -> mp_status {
      int s = 0;
      if (fused) {
        for (; s + 1 < nu; s += 2) {
          CKS(fsweep((const float *)x, lv.t32, c0, first_zero && s == 0));
          CKS(fsweep(lv.t32, (float *)x, c0, 0));
        }
      }
      for (; s < nu; ++s) {
        CKS(sweep(c0, first_zero && s == 0));
        CKS(sweep(1 - c0, 0));
      }
      return MP_OK;
    };
    CKS(smooth(lv.nu1, 0, 1));
    if constexpr (sizeof(T) == 4) {
      if (lv.d.nx % 4 == 0)
        LAUNCH_PDL(hd, K_RESTR32, l, 4.625 * nl * sz, k_resid_restrict_h4,
                   dim3((lv.d.nx / 4 + BX - 1) / BX, (lc.d.ny + BY - 1) / BY, lc.d.nz), kBlock,
                   0, x, rhs, lv.bx16, lv.by16, lv.bz16, (const __half *)lv.dd16, 1.f / hd->fs16,
                   lv.d, LV<T>::b(lc), lc.d);
      else
        LAUNCH_PDL(hd, K_RESTR32, l, 4.625 * nl * sz, k_resid_restrict_h, cell_grid(lc.d),
                   kBlock, 0, x, rhs, lv.bx16, lv.by16, lv.bz16, (const __half *)lv.dd16,
                   1.f / hd->fs16, lv.d, LV<T>::b(lc), lc.d);
    } else
      LAUNCH_PDL(hd, kid<T>(K_RESTR64, K_RESTR32), l, 6.125 * nl * sz, k_resid_restrict<T>,
                 cell_grid(lc.d), kBlock, 0, x, rhs, bx, by, bz, diag, lv.d, LV<T>::b(lc), lc.d);
    CKS(launch_ok());
    CKS(vcycle<T>(hd, l + 1, LV<T>::b(lc), LV<T>::e(lc)));
    constexpr int W = 16 / sizeof(T);
    if (lv.d.nx % (2 * W) == 0)
      LAUNCH_PDL(hd, kid<T>(K_PROL64, K_PROL32), l, 2.125 * nl * sz, k_prolong_vec<T>,
                 dim3((lv.d.nx / W + BX - 1) / BX, (lv.d.ny + BY - 1) / BY, lv.d.nz), kBlock, 0,
                 x, LV<T>::e(lc), lv.d, lc.d);
    else
      LAUNCH_PDL(hd, kid<T>(K_PROL64, K_PROL32), l, 2.125 * nl * sz, k_prolong<T>,
                 cell_grid(lv.d), kBlock, 0, x, LV<T>::e(lc), lv.d, lc.d);
    CKS(smooth(lv.nu2, 1, 0));
  }
  return launch_ok();
}

void destroy_graphs(mp_poisson *hd) {
  for (auto &g : hd->graphs) cudaGraphExecDestroy(g.exec);
  hd->graphs.clear();
}

// A whole V-cycle from the finest level.  Without per-launch profiling it is
// captured once into a CUDA graph (per precision and buffer pair) and
// replayed: the cycle is a fixed sequence of ~100 launches, most of them on
// small coarse levels where launch latency, not bandwidth, sets the time.
template <typename T>
mp_status run_vcycle(mp_poisson *hd, const T *rhs, T *x) {
  if (hd->prof_on) return vcycle<T>(hd, 0, rhs, x);
  mp_poisson::Graph *g = nullptr;
  for (auto &e : hd->graphs)
    if (e.type == (int)sizeof(T) && e.rhs == rhs && e.x == x) g = &e;
  if (!g) {
    cudaStream_t saved = hd->st;
    hd->st = hd->cap;
    hd->capturing = true;
    hd->cap_ids.clear();
    hd->cap_levels.clear();
    cudaError_t e0 = cudaStreamBeginCapture(hd->cap, cudaStreamCaptureModeThreadLocal);
    mp_status s = e0 == cudaSuccess ? vcycle<T>(hd, 0, rhs, x) : MP_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(hd->cap, &graph);
    hd->st = saved;
    hd->capturing = false;
    if (s != MP_OK || e0 != cudaSuccess || e1 != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return s != MP_OK ? s : MP_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      return MP_ERR_CUDA;
    }
    hd->graphs.push_back(mp_poisson::Graph{(int)sizeof(T), rhs, x, exec, hd->cap_ids,
                                           hd->cap_levels});
    g = &hd->graphs.back();
  }
  CK(cudaGraphLaunch(g->exec, hd->st));
  for (size_t k = 0; k < g->ids.size(); ++k) hd->prof[g->ids[k]][g->levels[k]].launches++;
  return MP_OK;
}

bool bad(double v) { return !std::isfinite(v); }

// ------------------------------------------------ deflation (mp_deflate.cuh)
// bytes of the fixed-point sums of m components (two words per replica)
size_t defl_acc_bytes(int m) { return (size_t)m * DEFL_REP * 2 * sizeof(unsigned long long); }

// Gas components of the current geometry, their boundary band and E = Z^T A Z.
// Deflation is off for this geometry (defl_m = 0) when there is no gas, more
// than DEFL_MAX components, or a labelling loop ran out of its bound.
mp_status deflation_setup(mp_poisson *hd) {
  Level &l0 = hd->L[0];
  const size_t n = hd->n;
  hd->defl_m = 0;
  hd->defl_nband = 0;
  if (n >= ((size_t)1 << 31)) return MP_OK;  // 32-bit cell indices
  // the band sums form E = Z^T A Z from the face arrays, which do not hold the
  // outflow faces: deflation is for periodic and wall boundaries
  if (hd->outflow) return MP_OK;
  const int nblk = (int)((n + BAND_CELLS - 1) / BAND_CELLS);
  // dint: [0] components (roots), [1] band cells, [2] labelling bound exceeded
  CK(cudaMemsetAsync(hd->dint, 0, 4 * sizeof(int), hd->st));
  const dim3 ct_grid((l0.d.nx + CT_X - 1) / CT_X, (l0.d.ny + CT_Y - 1) / CT_Y,
                     (l0.d.nz + CT_Z - 1) / CT_Z);
  const int lim = hd->opts.label_limit;
  LAUNCH(hd, K_DEFL_LABEL, 0, n * 12.0, k_ccl_tile, ct_grid, CT_THREADS, hd->phi, hd->lab, l0.d,
         hd->dint + 2, lim, hd->troots, hd->dint + 3, hd->tcap);
  LAUNCH(hd, K_DEFL_LABEL, 0, n * 4.0, k_ccl_faces, ct_grid, CT_THREADS, hd->lab, l0.d, hd->per,
         hd->dint + 2, lim);
  LAUNCH(hd, K_DEFL_LABEL, 0, hd->tcap * 8.0, k_ccl_flatten_roots, VEC_BLOCKS, VEC_THREADS, hd->lab,
         (const int *)hd->troots, (const int *)(hd->dint + 3), hd->tcap, hd->dint + 2, hd->roots,
         hd->dint, lim);
  LAUNCH(hd, K_DEFL_LABEL, 0, n * 8.0, k_ccl_flatten, VEC_BLOCKS, VEC_THREADS, hd->lab, n, hd->dint + 2,
         hd->roots, hd->dint, lim, (const int *)(hd->dint + 3), hd->tcap);
  LAUNCH(hd, K_DEFL_LABEL, 0, DEFL_MAX * 8.0, k_rank_roots, 1, 1024, hd->roots, hd->dint, hd->comp);
  LAUNCH(hd, K_DEFL_LABEL, 0, n * 12.0, k_comp_from_roots, VEC_BLOCKS, VEC_THREADS, hd->lab, hd->comp,
         n);
  CK(cudaMemcpyAsync(hd->hint, hd->dint, 4 * sizeof(int), cudaMemcpyDeviceToHost, hd->st));
  CK(cudaStreamSynchronize(hd->st));
  const int m = hd->hint[0];
  if (hd->hint[2] != 0 || m <= 0 || m > DEFL_MAX) return MP_OK;
  LAUNCH(hd, K_DEFL_LABEL, 0, n * 5.0, k_band_count, nblk, BAND_THREADS, hd->comp, l0.d, n, hd->cnt,
         hd->bflag);
  LAUNCH(hd, K_DEFL_LABEL, 0, nblk * 8.0, k_scan_counts, 1, SCAN_THREADS, hd->cnt, nblk, hd->dint + 1);
  LAUNCH(hd, K_DEFL_LABEL, 0, n * 1.0, k_band_assign, nblk, BAND_THREADS, hd->bflag, n, hd->cnt,
         hd->band);
  CK(cudaMemcpyAsync(hd->hint, hd->dint, 4 * sizeof(int), cudaMemcpyDeviceToHost, hd->st));
  CK(cudaStreamSynchronize(hd->st));
  const int nband = hd->hint[1];
  if (nband <= 0) return MP_OK;
  // E_jj = -sum of the boundary faces (fixed point: |E| <= 6 beta_max nband)
  const double escale = std::ldexp(1.0, 60) / (6.0 * hd->beta_max * (double)nband + 1.0);
  CK(cudaMemsetAsync(hd->acc_a, 0, defl_acc_bytes(m), hd->st));
  LAUNCH(hd, K_DEFL, 0, nband * 60.0, k_defl_E<double>, VEC_BLOCKS, VEC_THREADS, hd->band, nband,
         hd->comp, l0.bx, l0.by, l0.bz, l0.d, hd->acc_a, escale);
  LAUNCH(hd, K_DEFL, 0, m * 8.0, k_defl_einv, (m + 255) / 256, 256, m, hd->acc_a, escale,
         hd->einv);
  CKS(launch_ok());
  hd->defl_m = m;
  hd->defl_nband = nband;
  return MP_OK;
}

bool defl_active(const mp_poisson *hd) {
  return hd->opts.deflate && hd->opts.method == 0 && hd->defl_m > 0;
}

// Z^T b of the current right-hand side (fixed point, |b_c| <= ||b||).  Called
// at the start of a deflated solve: also clears the per-projection sums and
// the band maximum, which every projection leaves zeroed for the next.
mp_status defl_ztb(mp_poisson *hd) {
  const int m = hd->defl_m;
  hd->ztb_scale = std::ldexp(1.0, 60) / ((double)hd->n * std::max(hd->bnorm, 1e-300));
  CK(cudaMemsetAsync(hd->acc_ztb, 0, defl_acc_bytes(m), hd->st));
  CK(cudaMemsetAsync(hd->acc_a, 0, defl_acc_bytes(m), hd->st));
  CK(cudaMemsetAsync(hd->acc_b, 0, defl_acc_bytes(m), hd->st));
  CK(cudaMemsetAsync(hd->dmax, 0, sizeof(unsigned long long), hd->st));
  LAUNCH(hd, K_DEFL_DOT, 0, hd->n * 12.0, k_defl_zt<double>, VEC_BLOCKS, VEC_THREADS, hd->comp, hd->b,
         hd->n, hd->acc_ztb, hd->ztb_scale);
  return launch_ok();
}

// coef = E^-1 (A Z)^T v on the band (minus_ztb: coef = E^-1 (Z^T b - (A Z)^T v),
// i.e. for v = x, E^-1 Z^T (b - A x))
template <typename T, typename F>
mp_status defl_coef(mp_poisson *hd, const T *v, const F *bx, const F *by, const F *bz,
                    bool with_ztb) {
  Level &l0 = hd->L[0];
  const int m = hd->defl_m, nb = hd->defl_nband;
  unsigned long long *acc = with_ztb ? hd->acc_b : hd->acc_a;
  LAUNCH(hd, K_DEFL, 0, nb * (double)sizeof(T), k_defl_maxabs<T>, VEC_BLOCKS, VEC_THREADS,
         hd->band, nb, v, hd->dmax);
  // k_defl_azt and k_defl_coef follow the kernel launched just before them:
  // programmatic serialization (both wait for their predecessor first)
  auto kazt = k_defl_azt<T, F>;
  LAUNCH_PDL(hd, K_DEFL, 0, nb * (7.0 * sizeof(T) + 3.0 * sizeof(F) + 28.0), kazt, VEC_BLOCKS,
             VEC_THREADS, 0, hd->band, nb, hd->comp, bx, by, bz, l0.d, v,
             (const unsigned long long *)hd->dmax, hd->beta_max, acc, hd->dscale);
  if (with_ztb)
    LAUNCH_PDL(hd, K_DEFL, 0, m * 16.0, k_defl_coef, (m + 255) / 256, 256, 0, m, hd->acc_ztb,
               (const double *)nullptr, hd->ztb_scale, 0, acc, (const double *)hd->dscale,
               (const double *)hd->einv, hd->coef, hd->coef32, hd->dmax);
  else
    LAUNCH_PDL(hd, K_DEFL, 0, m * 16.0, k_defl_coef, (m + 255) / 256, 256, 0, m, acc,
               (const double *)hd->dscale, 0.0, 1, (unsigned long long *)nullptr,
               (const double *)nullptr, (const double *)hd->einv, hd->coef, hd->coef32,
               hd->dmax);
  return launch_ok();
}

// v -= A Z coef on the band
template <typename T, typename F>
mp_status defl_sub(mp_poisson *hd, T *v, const F *bx, const F *by, const F *bz) {
  Level &l0 = hd->L[0];
  const int nb = hd->defl_nband;
  auto ksub = k_defl_sub_aw<T, F>;
  LAUNCH(hd, K_DEFL, 0, nb * (2.0 * sizeof(T) + 3.0 * sizeof(F) + 28.0), ksub, VEC_BLOCKS,
         VEC_THREADS, hd->band, nb, hd->comp, bx, by, bz, l0.d, hd->coef, v);
  return launch_ok();
}

// x += Z E^-1 Z^T (b - A x): the deflation correction of the final iterate
mp_status defl_finish(mp_poisson *hd, double *x) {
  Level &l0 = hd->L[0];
  CKS((defl_coef<double, double>(hd, x, l0.bx, l0.by, l0.bz, true)));
  LAUNCH(hd, K_DEFL_DOT, 0, hd->n * 12.0, k_defl_add_z, VEC_BLOCKS, VEC_THREADS, x, hd->comp, hd->n,
         hd->coef);
  return launch_ok();
}

// The residuals deflated CG starts from, for the guess p and for the zero
// guess: ||P (bt - At p)|| and ||P bt|| (P = I - At Z E^-1 Z^T), formed in FP64
// in the scratch vector hd->z.  Uses hd->q as scratch too.
mp_status defl_guess_residuals(mp_poisson *hd, const double *p, double *rguess, double *rzero) {
  Level &l0 = hd->L[0];
  const size_t n = hd->n;
  CKS(defl_ztb(hd));
  LAUNCH(hd, K_RESID64, 0, n * 56.0, k_residual<double>, zgrid(l0.d), kBlock, p, hd->b, hd->z,
         l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial, 0);
  CKS((defl_coef<double, double>(hd, p, l0.bx, l0.by, l0.bz, true)));
  CKS((defl_sub<double, double>(hd, hd->z, l0.bx, l0.by, l0.bz)));
  LAUNCH(hd, K_DOT64, 0, n * 16.0, k_dot<double>, VEC_BLOCKS, VEC_THREADS, hd->z, hd->z, n,
         hd->partial);
  CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_TMP));
  CKS(read_scalars(hd));
  *rguess = std::sqrt(hd->scal_h[S_TMP]);
  // zero guess: coef = E^-1 Z^T bt, P bt = bt - At Z coef
  const int m = hd->defl_m;
  LAUNCH(hd, K_DEFL, 0, m * 16.0, k_defl_coef, (m + 255) / 256, 256, m, hd->acc_ztb,
         (const double *)nullptr, hd->ztb_scale, 0, (unsigned long long *)nullptr,
         (const double *)nullptr, hd->einv, hd->coef, hd->coef32, hd->dmax);
  CK(cudaMemcpyAsync(hd->z, hd->b, n * sizeof(double), cudaMemcpyDeviceToDevice, hd->st));
  CKS((defl_sub<double, double>(hd, hd->z, l0.bx, l0.by, l0.bz)));
  LAUNCH(hd, K_DOT64, 0, n * 16.0, k_dot<double>, VEC_BLOCKS, VEC_THREADS, hd->z, hd->z, n,
         hd->partial);
  CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_TMP));
  CKS(read_scalars(hd));
  *rzero = std::sqrt(hd->scal_h[S_TMP]);
  return MP_OK;
}

// z <- P^T z = z - Z E^-1 (A Z)^T z after the V-cycle, fused with the partial
// sums of r . z (the A-DEF2 form of deflated PCG: every search direction is
// A-orthogonal to the components, so the iteration needs no projection of A d)
template <typename T, typename F>
mp_status defl_rz(mp_poisson *hd, const T *r, T *z, const F *bx, const F *by, const F *bz) {
  CKS((defl_coef<T, F>(hd, z, bx, by, bz, false)));
  const T *coef;
  if constexpr (sizeof(T) == 8)
    coef = hd->coef;
  else
    coef = hd->coef32;
  LAUNCH_PDL(hd, K_DEFL_DOT, 0, hd->n * (3.0 * sizeof(T) + 4.0), k_dot_zdefl<T>, VEC_BLOCKS,
             VEC_THREADS, 0, r, z, (const int *)hd->comp, coef, hd->n, hd->partial);
  return launch_ok();
}

// Preconditioned CG on At x = (rhs), starting from x with residual r already
// formed and scal[S_RR] = r.r.  Stops when sqrt(r.r) <= tol_abs or after
// maxit iterations.  hist (may be null) receives sqrt(r.r)/bnorm.
template <typename T>
mp_status pcg(mp_poisson *hd, T *x, T *r, T *z, T *dv, T *q, double tol_abs, int maxit,
              int *iters, std::vector<double> *hist, double hist_scale) {
  Level &l0 = hd->L[0];
  T *bx = LV<T>::bx(l0), *by = LV<T>::by(l0), *bz = LV<T>::bz(l0), *diag = LV<T>::diag(l0);
  size_t n = hd->n;
  const double nsz = (double)n * sizeof(T);
  // deflated CG (FP64, A-DEF2 form): r <- P r = b - A (x + Z c) (c = E^-1 Z^T
  // (b - A x), the correction itself deferred), z <- P^T M r every iteration,
  // finish with x += Z E^-1 Z^T (b - A x), which includes c
  const bool defl = sizeof(T) == 8 && defl_active(hd);
  if (defl) {
    CKS(defl_ztb(hd));
    CKS((defl_coef<T, T>(hd, x, bx, by, bz, true)));
    CKS((defl_sub<T, T>(hd, r, bx, by, bz)));
    LAUNCH(hd, kid<T>(K_DOT64, K_DOT32), 0, 2.0 * nsz, k_dot<T>, VEC_BLOCKS, VEC_THREADS, r, r, n,
           hd->partial);
    CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_RR));
  }
  int it = 0;
  mp_status st = MP_OK;
  CKS(read_scalars(hd));
  double rn = std::sqrt(hd->scal_h[S_RR]);
  while (true) {
    if (bad(rn)) return MP_ERR_DIVERGED;
    if (rn <= tol_abs) break;
    if (it >= maxit) {
      st = MP_ERR_NOT_CONVERGED;
      break;
    }
    CKS(run_vcycle<T>(hd, r, z));
    if (defl)
      CKS((defl_rz<T, T>(hd, r, z, bx, by, bz)));
    else
      LAUNCH(hd, kid<T>(K_DOT64, K_DOT32), 0, 2.0 * nsz, k_dot<T>, VEC_BLOCKS, VEC_THREADS, r, z,
             n, hd->partial);
    CKS(reduce(hd, VEC_BLOCKS, it == 0 ? OP_STORE : OP_BETA, S_RZ));
    LAUNCH(hd, kid<T>(K_XPBY64, K_XPBY32), 0, (it == 0 ? 2.0 : 3.0) * nsz, k_xpby<T>, VEC_BLOCKS,
           VEC_THREADS, dv, z, n, hd->scal, it == 0);
    LAUNCH(hd, kid<T>(K_APPLY64, K_APPLY32), 0, (sizeof(T) == 8 ? 6.0 : 5.0) * nsz,
           k_apply_dot<T>, zgrid(l0.d), kBlock, dv, q, bx, by, bz, diag, (const T *)nullptr, l0.d,
           zper_of(l0.d),
           hd->partial);
    CKS(reduce(hd, zblocks(l0.d), OP_ALPHA, 0));
    LAUNCH(hd, kid<T>(K_AXPY64, K_AXPY32), 0, 6.0 * nsz, k_axpy2<T>, VEC_BLOCKS, VEC_THREADS, x,
           r, dv, q, n, hd->scal, hd->partial);
    CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_RR));
    ++it;
    CKS(read_scalars(hd));
    rn = std::sqrt(hd->scal_h[S_RR]);
    if (hist) hist->push_back(rn * hist_scale);
  }
  if (defl) CKS(defl_finish(hd, reinterpret_cast<double *>(x)));
  *iters = it;
  return st;
}

// r32 = fl32(P (bt - At p)) and its norm, deflation active.  The projection
// is formed in FP64 and rounded afterwards: near the components both bt - At p
// and A Z c are large, and rounding before the subtraction would leave their
// FP32 rounding error in the projected residual.  p_is_zero: p is taken as
// zero (not read), so bt - At p = bt off the band without the FP64 stencil.
// Needs defl_ztb of the current right-hand side.
mp_status defl_true_residual32(mp_poisson *hd, const double *p, int p_is_zero, double *rnorm) {
  Level &l0 = hd->L[0];
  const size_t n = hd->n;
  const int m = hd->defl_m, nb = hd->defl_nband;
  if (p_is_zero)  // coef = E^-1 Z^T bt
    LAUNCH(hd, K_DEFL, 0, m * 16.0, k_defl_coef, (m + 255) / 256, 256, m, hd->acc_ztb,
           (const double *)nullptr, hd->ztb_scale, 0, (unsigned long long *)nullptr,
           (const double *)nullptr, hd->einv, hd->coef, hd->coef32, hd->dmax);
  else
    CKS((defl_coef<double, double>(hd, p, l0.bx, l0.by, l0.bz, true)));
  LAUNCH(hd, K_RESIDMIX, 0, n * (p_is_zero ? 12.0 : 52.0), k_residual_mixed, zgrid(l0.d), kBlock,
         p, hd->b, hd->r32, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial,
         p_is_zero);
  LAUNCH(hd, K_DEFL, 0, nb * 120.0, k_defl_resid_band, VEC_BLOCKS, VEC_THREADS, hd->band, nb,
         hd->comp, l0.bx, l0.by, l0.bz, l0.diag, l0.d, hd->coef,
         p_is_zero ? (const double *)nullptr : p, hd->b, hd->r32);
  LAUNCH(hd, K_DOT32, 0, 4.0 * n, k_dot<float>, VEC_BLOCKS, VEC_THREADS, hd->r32, hd->r32, n,
         hd->partial);
  CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_RR));
  CKS(read_scalars(hd));
  *rnorm = std::sqrt(hd->scal_h[S_RR]);
  return MP_OK;
}

// Mixed-precision PCG with reliable updates.  The Krylov iteration (V-cycle
// preconditioner, operator, vector updates) runs in FP32 on a correction e32
// and residual r32.  Whenever the recurrence residual has fallen by
// inner_rtol since the last true residual (or after inner_max iterations),
// the correction is added to the FP64 solution p and r32 is replaced by the
// true FP64 residual bt - At p (rounded to FP32).  The search direction is
// kept across replacements (no restart), so the iteration count stays close
// to that of FP64 PCG while every stencil sweep moves 4-byte values.
// On entry r32 holds the true residual of p with norm rn; p_zero: p is zero;
// r_projected: r32 is already the deflated residual (rn its norm) and Z^T bt
// is formed.
mp_status pcg_mixed(mp_poisson *hd, double *p, double rn, double tol_abs, int maxit, int *iters,
                    int *outer, std::vector<double> *hist, double inv_b, bool p_zero,
                    bool r_projected) {
  Level &l0 = hd->L[0];
  const mp_opts &o = hd->opts;
  const size_t n = hd->n;
  const double nsz = (double)n * sizeof(float);
  float *e = hd->e32, *r = hd->r32, *z = hd->z32, *dv = hd->d32, *q = hd->q32;
  int it = 0, nrep = 0, since = 0;
  mp_status st = MP_OK;
  // deflated (A-DEF2 form): every true residual is projected, r32 = fl32(P (bt -
  // At p)), with Z^T (bt - At p) = Z^T bt - (At Z)^T p from FP64 p; after every
  // V-cycle z <- P^T z in FP32; the exit adds Z E^-1 Z^T (bt - At p) to p
  const bool defl = defl_active(hd);
  auto project_true = [&](double &rnorm, int p_is_zero) -> mp_status {
    return defl_true_residual32(hd, p, p_is_zero, &rnorm);
  };
  if (defl && !r_projected) {
    CKS(defl_ztb(hd));
    CKS(project_true(rn, p_zero ? 1 : 0));
  }
  double rn_rep = rn, rec = rn;
  CK(cudaMemsetAsync(e, 0, n * sizeof(float), hd->st));
  while (true) {
    if (since > 0 && (rec <= std::fmax(o.inner_rtol * rn_rep, 0.5 * tol_abs) ||
                      since >= o.inner_max || it >= maxit)) {
      // reliable update: p += e32 (e32 = 0), r32 = bt - At p from FP64
      LAUNCH(hd, K_ADDF32, 0, n * 24.0, k_add_f32, VEC_BLOCKS, VEC_THREADS, p, e, n);
      if (defl) {
        CKS(project_true(rn, 0));
      } else {
        LAUNCH(hd, K_RESIDMIX, 0, n * 52.0, k_residual_mixed, zgrid(l0.d), kBlock, p, hd->b, r,
               l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial, 0);
        CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
        CKS(read_scalars(hd));
        rn = std::sqrt(hd->scal_h[S_RR]);
      }
      rn_rep = rec = rn;
      since = 0;
      ++nrep;
      if (hist) hist->push_back(rn * inv_b);
    }
    if (bad(rec)) { st = MP_ERR_DIVERGED; break; }
    if (since == 0 && rn <= tol_abs) break;  // converged on a true residual
    if (it >= maxit) { st = MP_ERR_NOT_CONVERGED; break; }
    CKS(run_vcycle<float>(hd, r, z));
    if (defl)
      CKS((defl_rz<float, float>(hd, r, z, l0.bx32, l0.by32, l0.bz32)));
    else
      LAUNCH(hd, K_DOT32, 0, 2.0 * nsz, k_dot<float>, VEC_BLOCKS, VEC_THREADS, r, z, n,
             hd->partial);
    // from here to the end of the iteration every launch follows a kernel:
    // programmatic serialization, each kernel waiting for its predecessor
    CKS(reduce_after(hd, VEC_BLOCKS, it == 0 ? OP_STORE : OP_BETA, S_RZ));
    const bool fused = l0.d.nx % 4 == 0;  // 16-byte rows
    if (fused) {
      // d_new = z + beta d in the operator's loads, stored to the other buffer
      const Dims dq = chunk_dims(l0.d);
      float *dnew = dv == hd->d32 ? hd->d32b : hd->d32;
      LAUNCH_PDL(hd, K_APPLY32, 0, (it == 0 ? 6.0 : 7.0) * nsz, k_apply_dot4<true>, zgrid(dq),
                 kBlock, 0, (const float *)dv, q, (const float *)l0.bx32,
                 (const float *)l0.by32, (const float *)l0.bz32, (const float *)l0.dd32, l0.d,
                 zper_of(dq), hd->partial, (const float *)z, dnew, (const double *)hd->scal,
                 it == 0 ? 1 : 0);
      CKS(reduce_after(hd, zblocks(dq), OP_ALPHA, 0));
      dv = dnew;
    } else {
      LAUNCH(hd, K_XPBY32, 0, (it == 0 ? 2.0 : 3.0) * nsz, k_xpby<float>, VEC_BLOCKS, VEC_THREADS,
             dv, z, n, hd->scal, it == 0);
      LAUNCH(hd, K_APPLY32, 0, 5.0 * nsz, k_apply_dot<float>, zgrid(l0.d), kBlock, dv, q,
             l0.bx32, l0.by32, l0.bz32, (float *)nullptr, (const float *)l0.dd32, l0.d,
             zper_of(l0.d), hd->partial);
      CKS(reduce(hd, zblocks(l0.d), OP_ALPHA, 0));
    }
    LAUNCH_PDL(hd, K_AXPY32, 0, 6.0 * nsz, k_axpy2<float>, VEC_BLOCKS, VEC_THREADS, 0, e, r,
               (const float *)dv, (const float *)q, n, (const double *)hd->scal, hd->partial);
    CKS(reduce_after(hd, VEC_BLOCKS, OP_STORE, S_RR));
    ++it;
    ++since;
    CKS(read_scalars(hd));
    rec = std::sqrt(hd->scal_h[S_RR]);
  }
  if (defl && st != MP_ERR_DIVERGED) CKS(defl_finish(hd, p));
  *iters = it;
  *outer = nrep;
  return st;
}

// Stationary V-cycle iteration: x += V(r); r = bt - At x.
template <typename T>
mp_status stationary(mp_poisson *hd, T *x, const T *bt, T *r, T *z, double tol_abs, int maxit,
                     int *iters, std::vector<double> *hist, double hist_scale) {
  Level &l0 = hd->L[0];
  T *bx = LV<T>::bx(l0), *by = LV<T>::by(l0), *bz = LV<T>::bz(l0), *diag = LV<T>::diag(l0);
  int it = 0;
  CKS(read_scalars(hd));
  double rn = std::sqrt(hd->scal_h[S_RR]);
  while (true) {
    if (bad(rn)) return MP_ERR_DIVERGED;
    if (rn <= tol_abs) break;
    if (it >= maxit) {
      *iters = it;
      return MP_ERR_NOT_CONVERGED;
    }
    CKS(run_vcycle<T>(hd, r, z));
    const double nsz = (double)hd->n * sizeof(T);
    LAUNCH(hd, kid<T>(K_ADD64, K_ADD32), 0, 3.0 * nsz, k_add<T>, VEC_BLOCKS, VEC_THREADS, x, z,
           hd->n);
    LAUNCH(hd, kid<T>(K_RESID64, K_RESID32), 0, 7.0 * nsz, k_residual<T>, zgrid(l0.d), kBlock,
           x, bt, r, bx, by, bz, diag, l0.d, zper_of(l0.d), hd->partial, 0);
    CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
    ++it;
    CKS(read_scalars(hd));
    rn = std::sqrt(hd->scal_h[S_RR]);
    if (hist) hist->push_back(rn * hist_scale);
  }
  *iters = it;
  return MP_OK;
}

// mean removal of a device FP64 vector (gauge)
mp_status remove_mean(mp_poisson *hd, double *x) {
  LAUNCH(hd, K_SUM, 0, hd->n * 8.0, k_sum<double>, VEC_BLOCKS, VEC_THREADS, x, hd->n, hd->partial);
  CKS(reduce(hd, VEC_BLOCKS, OP_MEAN, 0, (double)hd->n));
  LAUNCH(hd, K_SUBMEAN, 0, hd->n * 16.0, k_sub_mean, VEC_BLOCKS, VEC_THREADS, x, hd->n, hd->scal,
         nullptr);
  return launch_ok();
}

// bt (already holding h^2 rhs + Jt with block sums in partial, np blocks)
// -> subtract mean, store ||bt||^2 in S_BB
// With an outflow side the operator is nonsingular: b keeps its mean and only
// ||bt||^2 is formed.
mp_status finish_rhs(mp_poisson *hd, int np) {
  if (hd->outflow) {
    LAUNCH(hd, K_DOT64, 0, hd->n * 8.0, k_dot<double>, VEC_BLOCKS, VEC_THREADS, hd->b, hd->b,
           hd->n, hd->partial);
    CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_BB));
    return launch_ok();
  }
  CKS(reduce(hd, np, OP_MEAN, 0, (double)hd->n));
  LAUNCH(hd, K_SUBMEAN, 0, hd->n * 16.0, k_sub_mean, VEC_BLOCKS, VEC_THREADS, hd->b, hd->n,
         hd->scal, hd->partial);
  CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_BB));
  return launch_ok();
}

mp_status assemble_rhs(mp_poisson *hd, const double *rhs) {
  LAUNCH(hd, K_ASSEMBLE, 0, hd->n * 24.0, k_assemble, VEC_BLOCKS, VEC_THREADS, rhs, hd->Jt, hd->b,
         hd->n, hd->h * hd->h, hd->partial);
  CKS(launch_ok());
  return finish_rhs(hd, VEC_BLOCKS);
}

mp_status assemble_rhs_u(mp_poisson *hd, const double *ux, const double *uy, const double *uz) {
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_ASSEMBLE_U, 0, hd->n * 40.0, k_assemble_u, zgrid(l0.d), kBlock, ux, uy, uz,
         hd->Jt, hd->b, l0.d, zper_of(l0.d), 0, hd->h, hd->partial);
  CKS(launch_ok());
  return finish_rhs(hd, zblocks(l0.d));
}

// z-slabs of the host-buffer step: groups of whole z-blocks of zgrid(l0)
struct Slabs {
  int count = 1, per = 1, zper = 1, zb = 1;  // slabs, z-blocks per slab, planes per z-block
  int kb_lo(int s) const { return s * per; }
  int kb_hi(int s) const { return std::min(zb, (s + 1) * per); }
};
Slabs slabs_of(const Dims &d) {
  Slabs q;
  q.zper = zper_of(d);
  q.zb = (int)zgrid(d).z;
  q.count = std::min(q.zb, MAX_SLABS);
  q.per = (q.zb + q.count - 1) / q.count;
  q.count = (q.zb + q.per - 1) / q.per;
  return q;
}

mp_status diag_fields(mp_poisson *hd, int mode);

// Solve At p = bt (bt in hd->b, S_BB set).  p: device FP64, in/out.
mp_status solve_assembled(mp_poisson *hd, double *p, double tol, std::vector<double> *hist) {
  Level &l0 = hd->L[0];
  const mp_opts &o = hd->opts;
  CKS(read_scalars(hd));
  hd->bnorm = std::sqrt(hd->scal_h[S_BB]);
  hd->stats = mp_stats{};
  hd->stats.levels = (int)hd->L.size();
  hd->stats.coarse_n = hd->nc;
  hd->stats.components = defl_active(hd) ? hd->defl_m : 0;
  if (o.initial_guess == 2 && !hd->net) return MP_ERR_NO_NET;
  if (o.initial_guess == 2 && hd->outflow) return MP_ERR_INVALID_ARG;  // walls/periodic only
  const int need = o.precision == 0 ? 1 : 2;
  if ((hd->diag_mode & need) != need) CKS(diag_fields(hd, need));
  int zero = o.initial_guess == 0;
  if (zero) CK(cudaMemsetAsync(p, 0, hd->n * sizeof(double), hd->st));
  if (hd->bnorm == 0.0) {
    CK(cudaMemsetAsync(p, 0, hd->n * sizeof(double), hd->st));
    CK(cudaStreamSynchronize(hd->st));
    if (hist) hist->push_back(0.0);
    return MP_OK;
  }
  // the residual of a learned guess, once formed, is the solve's initial
  // residual; r_projected: r32 and S_RR already hold the deflated residual of
  // the zero guess (and Z^T bt is formed) after a rejected guess
  bool have_r = false, r_projected = false;
  if (o.initial_guess == 2) {
    // learned guess: features from phi and the assembled rhs, network output q
    // (the shape), scaled by the energy-optimal alpha = (q . bt) / (q . At q),
    // which minimises the A-norm error of alpha q; kept per net_check
    double s = 1.0;
    CK(cudaStreamSynchronize(hd->st));
    CKS(mp_net_set_stream(hd->net, hd->st));
    CKS(mp_net_features_at(hd->net, hd->net_factor, hd->phi, hd->b, hd->h, 1.0, &s));
    CKS(mp_net_forward(hd->net, nullptr));
    const mp_bc nbc[3] = {(hd->per & 1) ? MP_BC_PERIODIC : MP_BC_NEUMANN,
                          (hd->per & 2) ? MP_BC_PERIODIC : MP_BC_NEUMANN,
                          (hd->per & 4) ? MP_BC_PERIODIC : MP_BC_NEUMANN};
    CKS(mp_net_pressure_at(hd->net, hd->net_factor, nbc, 1.0, p));
    if (o.precision == 1 && l0.d.nx % 4 == 0) {
      // q . At q from the FP32 operator on fl32(q): alpha is a scale factor,
      // and 1e-7 relative is ample (an FP64 operator pass is FP64-rate bound)
      LAUNCH(hd, K_RESIDMIX, 0, hd->n * 12.0, k_to_f32_norm, VEC_BLOCKS, VEC_THREADS, p, hd->z32,
             hd->n, hd->partial);
      const Dims dq = chunk_dims(l0.d);
      LAUNCH(hd, K_APPLY32, 0, hd->n * 20.0, k_apply_dot4<false>, zgrid(dq), kBlock,
             (const float *)hd->z32, hd->q32, l0.bx32, l0.by32, l0.bz32, (const float *)l0.dd32,
             l0.d, zper_of(dq), hd->partial, (const float *)nullptr, (float *)nullptr,
             (const double *)nullptr, 0);
      CKS(reduce(hd, zblocks(dq), OP_STORE, S_TMP));
    } else {
      LAUNCH(hd, K_APPLY64, 0, hd->n * 48.0, k_apply_dot<double>, zgrid(l0.d), kBlock, p, hd->q,
             l0.bx, l0.by, l0.bz, l0.diag, (const double *)nullptr, l0.d, zper_of(l0.d),
             hd->partial);
      CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_TMP));
    }
    LAUNCH(hd, K_DOT64, 0, hd->n * 16.0, k_dot<double>, VEC_BLOCKS, VEC_THREADS, p, hd->b, hd->n,
           hd->partial);
    CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_RZ));
    CKS(read_scalars(hd));
    double alpha = hd->scal_h[S_RZ] / hd->scal_h[S_TMP];
    if (!std::isfinite(alpha)) alpha = 0.0;
    LAUNCH(hd, K_SCALE, 0, hd->n * 16.0, k_scale, VEC_BLOCKS, VEC_THREADS, p, p, hd->n, alpha);
    double rnet = 0.0, rzero = hd->bnorm;
    const bool defl_mixed = defl_active(hd) && o.net_check == 0 && o.precision == 1;
    if (defl_mixed) {
      // deflated residuals of the guess and of the zero guess, the latter
      // last: a rejected guess leaves r32 = fl32(P bt), the start of the
      // zero-guess solve (mixed PCG forms a kept guess's again at its start)
      CKS(defl_ztb(hd));
      CKS(defl_true_residual32(hd, p, 0, &rnet));
      CKS(defl_true_residual32(hd, p, 1, &rzero));
    } else {
      if (o.precision == 0)
        LAUNCH(hd, K_RESID64, 0, hd->n * 56.0, k_residual<double>, zgrid(l0.d), kBlock, p, hd->b,
               hd->r, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial, 0);
      else
        LAUNCH(hd, K_RESIDMIX, 0, hd->n * 52.0, k_residual_mixed, zgrid(l0.d), kBlock, p,
               hd->b, hd->r32, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial, 0);
      CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
      CKS(read_scalars(hd));
      rnet = std::sqrt(hd->scal_h[S_RR]);
      if (defl_active(hd) && o.net_check == 0 && std::isfinite(rnet))
        CKS(defl_guess_residuals(hd, p, &rnet, &rzero));
    }
    hd->stats.net_relres = rnet / rzero;
    const bool keep = o.net_check == 0 ? rnet < rzero : alpha != 0.0;
    if (keep && std::isfinite(rnet)) {
      hd->stats.used_net = 1;
      have_r = true;
    } else {
      CK(cudaMemsetAsync(p, 0, hd->n * sizeof(double), hd->st));
      zero = 1;
      r_projected = defl_mixed && o.method == 0;  // (the stationary iteration is not deflated)
    }
  }
  double inv_b = 1.0 / hd->bnorm;
  double tol_abs = tol * hd->bnorm;
  mp_status st = MP_OK;
  int iters = 0;
  if (o.precision == 0) {
    if (!have_r) {
      LAUNCH(hd, K_RESID64, 0, hd->n * (zero ? 16.0 : 56.0), k_residual<double>, zgrid(l0.d),
             kBlock, p, hd->b, hd->r, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d),
             hd->partial, zero);
      CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
    }
    CKS(read_scalars(hd));
    hd->stats.r0 = std::sqrt(hd->scal_h[S_RR]) * inv_b;
    if (hist) hist->push_back(hd->stats.r0);
    if (o.method == 0)
      st = pcg<double>(hd, p, hd->r, hd->z, hd->dv, hd->q, tol_abs, o.max_iters, &iters, hist,
                       inv_b);
    else
      st = stationary<double>(hd, p, hd->b, hd->r, hd->z, tol_abs, o.max_iters, &iters, hist,
                              inv_b);
    hd->stats.iterations = iters;
    hd->stats.outer_steps = iters;
  } else {
    // FP64 iterative refinement around an FP32 inner solve
    if (!have_r && !r_projected) {
      LAUNCH(hd, K_RESIDMIX, 0, hd->n * (zero ? 12.0 : 52.0), k_residual_mixed, zgrid(l0.d),
             kBlock, p, hd->b, hd->r32, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d),
             hd->partial, zero);
      CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
    }
    CKS(read_scalars(hd));
    double rn = std::sqrt(hd->scal_h[S_RR]);
    hd->stats.r0 = r_projected ? 1.0 : rn * inv_b;  // the zero guess's residual is bt
    if (hist) hist->push_back(hd->stats.r0);
    int total = 0, outer = 0;
    while (true) {
      if (bad(rn)) { st = MP_ERR_DIVERGED; break; }
      if (rn <= tol_abs) { st = MP_OK; break; }
      if (total >= o.max_iters) { st = MP_ERR_NOT_CONVERGED; break; }
      if (o.method == 0) {
        // PCG with reliable updates (replaces the refinement loop)
        int pit = 0, pout = 0;
        st = pcg_mixed(hd, p, rn, tol_abs, o.max_iters, &pit, &pout, hist, inv_b, zero != 0,
                       r_projected);
        total = pit;
        outer = pout;
        if (st != MP_OK && st != MP_ERR_NOT_CONVERGED && st != MP_ERR_DIVERGED) return st;
        break;
      }
      // stationary: one FP32 V-cycle per FP64 refinement step
      CKS(run_vcycle<float>(hd, hd->r32, hd->e32));
      total += 1;
      ++outer;
      LAUNCH(hd, K_ADDF32, 0, hd->n * 24.0, k_add_f32, VEC_BLOCKS, VEC_THREADS, p, hd->e32,
             hd->n);
      LAUNCH(hd, K_RESIDMIX, 0, hd->n * 52.0, k_residual_mixed, zgrid(l0.d), kBlock, p, hd->b,
             hd->r32, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial, 0);
      CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
      CKS(read_scalars(hd));
      rn = std::sqrt(hd->scal_h[S_RR]);
      if (hist) hist->push_back(rn * inv_b);
    }
    hd->stats.iterations = total;
    hd->stats.outer_steps = outer;
  }
  if (st == MP_OK || st == MP_ERR_NOT_CONVERGED) {
    if (!hd->outflow) CKS(remove_mean(hd, p));  // gauge of the singular problem
    // final true FP64 residual of the returned p
    LAUNCH(hd, K_RESID64, 0, hd->n * 56.0, k_residual<double>, zgrid(l0.d), kBlock, p, hd->b,
           hd->r, l0.bx, l0.by, l0.bz, l0.diag, l0.d, zper_of(l0.d), hd->partial, 0);
    CKS(reduce(hd, zblocks(l0.d), OP_STORE, S_RR));
    CKS(read_scalars(hd));
    hd->stats.relres = std::sqrt(hd->scal_h[S_RR]) * inv_b;
  }
  return st;
}

bool valid_opts(const mp_opts &o) {
  return (o.precision == 0 || o.precision == 1) && (o.method == 0 || o.method == 1) &&
         o.initial_guess >= 0 && o.initial_guess <= 2 && o.max_iters >= 0 && o.nu1 >= 1 &&
         o.nu2 >= 1 && o.nu_growth >= 1 && o.nu_max >= 1 && o.inner_rtol > 0.0 &&
         o.inner_rtol < 1.0 && o.inner_max >= 1 && (o.net_check == 0 || o.net_check == 1) &&
         (o.deflate == 0 || o.deflate == 1) && (o.smoother == 0 || o.smoother == 1) &&
         o.label_limit >= 1 && (o.coarse_cluster == 0 || o.coarse_cluster == 1);
}

void apply_nu(mp_poisson *hd) {
  long f = 1;
  for (size_t l = 0; l < hd->L.size(); ++l) {
    hd->L[l].nu1 = (int)std::min<long>(hd->opts.nu_max, (long)hd->opts.nu1 * f);
    hd->L[l].nu2 = (int)std::min<long>(hd->opts.nu_max, (long)hd->opts.nu2 * f);
    f = std::min<long>(f * hd->opts.nu_growth, 1L << 20);
  }
}

// Per-level diagonal and face copies for the precisions in mode (bits: 1 = the
// FP64 smoother's 1/diag, 2 = the FP32 faces, 1/diag and FP16 faces); a solve
// in a precision whose arrays this geometry has not formed yet adds them.
mp_status diag_fields(mp_poisson *hd, int mode) {
  for (size_t l = 0; l < hd->L.size(); ++l) {
    Level &lv = hd->L[l];
    auto kd = mode == 1 ? k_diag<1> : (mode == 2 ? k_diag<2> : k_diag<3>);
    BndPlanes bp{};
    for (int q = 0; q < 6; ++q) bp.p[q] = lv.bnd[q];
    LAUNCH(hd, K_DIAG, (int)l, lv.n * (mode == 1 ? 48.0 : (mode == 2 ? 58.0 : 66.0)), kd,
           cell_grid(lv.d), kBlock, lv.bx, lv.by, lv.bz, lv.diag, lv.idiag, lv.bx32, lv.by32,
           lv.bz32, lv.idiag32, lv.bx16, lv.by16, lv.bz16, hd->fs16, lv.d, bp, lv.dd, lv.dd32,
           lv.dd16);
    CKS(launch_ok());
  }
  hd->diag_mode |= mode;
  return MP_OK;
}

mp_status geometry(mp_poisson *hd, const double *phi, double rho_l, double rho_g, double sigma) {
  if (!phi || !(rho_l > 0.0) || !(rho_g > 0.0) || !(sigma >= 0.0) || !std::isfinite(rho_l) ||
      !std::isfinite(rho_g) || !std::isfinite(sigma))
    return MP_ERR_INVALID_ARG;
  hd->rho_l = rho_l;
  hd->rho_g = rho_g;
  hd->sigma = sigma;
  Level &l0 = hd->L[0];
  CK(cudaMemcpyAsync(hd->phi, phi, hd->n * sizeof(double), cudaMemcpyDeviceToDevice, hd->st));
  const double n0 = (double)hd->n;
  LAUNCH(hd, K_CURV, 0, n0 * 16.0, k_curvature, cell_grid(l0.d), kBlock, hd->phi, hd->kap, l0.d,
         hd->h, hd->per);
  LAUNCH(hd, K_FACES, 0, n0 * 32.0, k_faces, cell_grid(l0.d), kBlock, hd->phi, l0.bx, l0.by,
         l0.bz, l0.d, rho_l, rho_g, 1.0 / rho_l, 1.0 / rho_g, hd->per);
  LAUNCH(hd, K_JUMP, 0, n0 * (hd->has_mdot ? 56.0 : 48.0), k_jump, cell_grid(l0.d), kBlock,
         hd->phi, hd->kap, l0.bx, l0.by, l0.bz, hd->Jt, l0.d, sigma, mdot_of(hd), rho_l, rho_g,
         hd->h);
  CKS(launch_ok());
  // faces never exceed 1 / min(rho): scale them so the largest sits in (2^13, 2^14]
  hd->beta_max = std::max(1.0 / rho_l, 1.0 / rho_g);
  hd->fs16 = (float)std::ldexp(1.0, 14 - (int)std::ceil(std::log2(hd->beta_max)));
  for (size_t l = 0; l < hd->L.size(); ++l) {
    Level &lv = hd->L[l];
    if (l > 0) {
      Level &lf = hd->L[l - 1];
      LAUNCH(hd, K_COARSEN, (int)l, lv.n * 120.0, k_coarsen_faces, cell_grid(lv.d), kBlock, lf.bx,
             lf.by, lf.bz, lf.d, lv.bx, lv.by, lv.bz, lv.d);
    }
  }
  if (hd->outflow) {  // outflow boundary faces of every level
    Level &f0 = hd->L[0];
    for (int q = 0; q < 6; ++q)
      if (f0.bnd[q]) {
        const int na = q < 2 ? f0.d.ny : f0.d.nx, nb = q < 4 ? f0.d.nz : f0.d.ny;
        LAUNCH(hd, K_FACES, 0, na * nb * 16.0, k_bnd_init, (na * nb + 255) / 256, 256, hd->phi,
               f0.bnd[q], f0.d, q, 1.0 / rho_l, 1.0 / rho_g);
      }
    for (size_t l = 1; l < hd->L.size(); ++l) {
      Level &lv = hd->L[l], &lf = hd->L[l - 1];
      for (int q = 0; q < 6; ++q)
        if (lv.bnd[q]) {
          const int na = q < 2 ? lv.d.ny : lv.d.nx, nb = q < 4 ? lv.d.nz : lv.d.ny;
          LAUNCH(hd, K_COARSEN, (int)l, na * nb * 40.0, k_bnd_coarsen, (na * nb + 255) / 256, 256,
                 lf.bnd[q], lv.bnd[q], na, nb);
        }
    }
    CKS(launch_ok());
  }
  hd->diag_mode = 0;
  CKS(diag_fields(hd, hd->opts.precision == 0 ? 1 : 2));
  Level &lc = hd->L.back();
  const int lcl = (int)hd->L.size() - 1;
  const double nc = (double)hd->nc;
  LAUNCH(hd, K_DENSE, lcl, nc * 2.0 * nc * 8.0, k_dense_build, (hd->nc + 127) / 128, 128, lc.bx,
         lc.by, lc.bz, lc.diag, hd->Maug, lc.d, hd->outflow == 0 ? 1 : 0);
  if (hd->nc <= GJ_SMEM_MAX)
    LAUNCH_SMEM(hd, K_GJ, lcl, nc * 3.0 * nc * 8.0, k_inverse_cols, hd->nc, 256,
                (size_t)(hd->nc + 1) * hd->nc * sizeof(double), hd->Maug, hd->Minv, hd->nc);
  else
    LAUNCH(hd, K_GJ, lcl, nc * 3.0 * nc * 8.0, k_gauss_jordan, 1, 1024, hd->Maug, hd->Minv,
           hd->nc);
  CKS(launch_ok());
  CKS(deflation_setup(hd));
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

// Grid of the fused sweep for every FP32 level it runs on (levels above the
// one-CTA tail, nx a multiple of 8), and the second iterate buffer.  The
// z-chunk count minimises (waves of resident CTAs) x (planes per chunk +
// the ~3.5 planes a chunk stages beyond its own).
mp_status fused_setup(mp_poisson *hd) {
  CK(cudaFuncSetAttribute(k_rbgs_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          FS_SMEM));
  CK(cudaFuncSetAttribute(k_rbgs_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          FS_SMEM));
  int dev = 0, sms = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rbgs_fused<false>, FS_THREADS,
                                                   FS_SMEM));
  const long slots = (long)std::max(1, sms) * std::max(1, per_sm);
  for (int l = 0; l < hd->tail32 && l < (int)hd->L.size() - 1; ++l) {
    Level &lv = hd->L[l];
    if (lv.d.nx % 8 != 0) continue;
    lv.ftx = (lv.d.nx + FS_TX - 1) / FS_TX;
    lv.fty = (lv.d.ny + FS_TY - 1) / FS_TY;
    const long tiles = (long)lv.ftx * lv.fty;
    double best = 0.0;
    for (int c = 1; c <= lv.d.nz; ++c) {
      if (tiles * c > (1L << 30)) break;
      const long waves = (tiles * c + slots - 1) / slots;
      const double cost = (double)waves * ((lv.d.nz + c - 1) / c + 3.5);
      if (lv.fchunk == 0 || cost < best - 1e-9) {
        best = cost;
        lv.fchunk = c;
      }
    }
    CKS(dalloc(hd, &lv.t32, lv.n));
  }
  return MP_OK;
}

// FP32 cluster tail (mp_ctail.cuh): the level above the one-CTA tail and every
// level below it in the shared memory of a CT_CTAS-CTA cluster, when every
// level's z-planes split evenly, the slabs fit and the device runs the cluster
mp_status ctail_setup(mp_poisson *hd) {
  hd->ctail32 = -1;
  const int nl = (int)hd->L.size(), top = hd->tail32 - 1;
  if (top < 0 || hd->tail32 >= nl - 1 || nl - top > CT_MAX_LEVELS) return MP_OK;
  if (hd->L.back().n > (size_t)CT_MAX_COARSE) return MP_OK;
  size_t floats = 0;
  for (int l = top; l < nl; ++l) {
    const Dims &d = hd->L[l].d;
    if (d.nz > CT_CTAS && d.nz % CT_CTAS != 0) return MP_OK;
    floats += ct_slab_floats(d, std::max(1, d.nz / CT_CTAS), hd->outflow != 0);
  }
  const size_t bytes = (floats + CT_MAX_COARSE) * sizeof(float);
  if (bytes > CT_SMEM_MAX) return MP_OK;
  if (cudaFuncSetAttribute(k_ctail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return MP_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CT_CTAS);
  cfg.blockDim = dim3(CTL_THREADS);
  cfg.dynamicSmemBytes = bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CT_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_ctail, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return MP_OK;
  }
  hd->ctail32 = top;
  hd->ctail_bytes = bytes;
  hd->ctail_scratch = (int)floats;
  return MP_OK;
}

mp_status create(mp_poisson *hd, mp_grid g, double h, const mp_bc bc[3]) {
  int dims[3] = {g.nx, g.ny, g.nz};
  hd->g = g;
  hd->h = h;
  hd->per = 0;
  hd->outflow = 0;
  for (int a = 0; a < 3; ++a) {
    if (bc[a] < MP_BC_PERIODIC || bc[a] > MP_BC_DIRICHLET_NEUMANN) return MP_ERR_INVALID_ARG;
    if (bc[a] == MP_BC_DIRICHLET || bc[a] == MP_BC_DIRICHLET_NEUMANN) hd->outflow |= 1 << (2 * a);
    if (bc[a] == MP_BC_DIRICHLET || bc[a] == MP_BC_NEUMANN_DIRICHLET)
      hd->outflow |= 1 << (2 * a + 1);
    if (dims[a] < 2 || dims[a] > (1 << 16)) return MP_ERR_INVALID_ARG;
    if (bc[a] == MP_BC_PERIODIC) {
      if (dims[a] & 1) return MP_ERR_INVALID_ARG;
      hd->per |= 1 << a;
    }
  }
  if (!(h > 0.0) || !std::isfinite(h)) return MP_ERR_INVALID_ARG;
  // hierarchy
  Dims d{g.nx, g.ny, g.nz};
  while (true) {
    Level lv;
    lv.d = d;
    lv.n = (size_t)d.nx * d.ny * d.nz;
    hd->L.push_back(lv);
    // halve while every dim is even and >= 4 and the level has more than 64 cells
    bool can = (d.nx % 2 == 0) && (d.ny % 2 == 0) && (d.nz % 2 == 0) && d.nx >= 4 && d.ny >= 4 &&
               d.nz >= 4 && (size_t)d.nx * d.ny * d.nz > 64;
    if (!can) break;
    d = Dims{d.nx / 2, d.ny / 2, d.nz / 2};
  }
  hd->nc = (int)hd->L.back().n;
  if (hd->nc > MAX_COARSE) return MP_ERR_INVALID_ARG;
  // a level that is smoothed must have even x (red-black pairs along x)
  for (size_t l = 0; l + 1 < hd->L.size(); ++l)
    if (hd->L[l].d.nx & 1) return MP_ERR_INVALID_ARG;
  hd->n = hd->L[0].n;
  size_t n = hd->n;
  for (size_t l = 0; l < hd->L.size(); ++l) {
    Level &lv = hd->L[l];
    CKS(dalloc(hd, &lv.bx, lv.n));
    CKS(dalloc(hd, &lv.by, lv.n));
    CKS(dalloc(hd, &lv.bz, lv.n));
    CKS(dalloc(hd, &lv.diag, lv.n));
    CKS(dalloc(hd, &lv.idiag, lv.n));
    CKS(dalloc(hd, &lv.bx32, lv.n));
    CKS(dalloc(hd, &lv.by32, lv.n));
    CKS(dalloc(hd, &lv.bz32, lv.n));
    CKS(dalloc(hd, &lv.idiag32, lv.n));
    CKS(dalloc(hd, &lv.bx16, lv.n));
    CKS(dalloc(hd, &lv.by16, lv.n));
    CKS(dalloc(hd, &lv.bz16, lv.n));
    if (l > 0) {
      CKS(dalloc(hd, &lv.b, lv.n));
      CKS(dalloc(hd, &lv.e, lv.n));
      CKS(dalloc(hd, &lv.b32, lv.n));
      CKS(dalloc(hd, &lv.e32, lv.n));
    }
    if (hd->outflow) {
      CKS(dalloc(hd, &lv.dd, lv.n));
      CKS(dalloc(hd, &lv.dd32, lv.n));
      CKS(dalloc(hd, &lv.dd16, lv.n));
      for (int q = 0; q < 6; ++q)
        if (hd->outflow & (1 << q)) {
          const size_t na = q < 2 ? lv.d.ny : lv.d.nx, nb = q < 4 ? lv.d.nz : lv.d.ny;
          CKS(dalloc(hd, &lv.bnd[q], na * nb));
        }
    }
  }
  CKS(dalloc(hd, &hd->phi, n));
  CKS(dalloc(hd, &hd->kap, n));
  CKS(dalloc(hd, &hd->Jt, n));
  CKS(dalloc(hd, &hd->b, n));
  CKS(dalloc(hd, &hd->r, n));
  CKS(dalloc(hd, &hd->z, n));
  CKS(dalloc(hd, &hd->dv, n));
  CKS(dalloc(hd, &hd->q, n));
  CKS(dalloc(hd, &hd->r32, n));
  CKS(dalloc(hd, &hd->e32, n));
  CKS(dalloc(hd, &hd->z32, n));
  CKS(dalloc(hd, &hd->d32, n));
  CKS(dalloc(hd, &hd->d32b, n));
  CKS(dalloc(hd, &hd->q32, n));
  CKS(dalloc(hd, &hd->ux, n));
  CKS(dalloc(hd, &hd->uy, n));
  CKS(dalloc(hd, &hd->uz, n));
  CKS(dalloc(hd, &hd->pst, n));
  CKS(dalloc(hd, &hd->Maug, (size_t)hd->nc * 2 * hd->nc));
  CKS(dalloc(hd, &hd->Minv, (size_t)hd->nc * hd->nc));
  hd->npart = std::max(std::max(cell_blocks(hd->L[0].d), zblocks(hd->L[0].d)), VEC_BLOCKS);
  CKS(dalloc(hd, &hd->partial, (size_t)hd->npart));
  CKS(dalloc(hd, &hd->scal, (size_t)S_COUNT));
  if (cudaMallocHost((void **)&hd->scal_h, S_COUNT * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    hd->scal_h = nullptr;
    return MP_ERR_OOM;
  }
  CK(cudaMemsetAsync(hd->scal, 0, S_COUNT * sizeof(double), hd->st));
  // deflation workspace
  const size_t nblk = (n + BAND_CELLS - 1) / BAND_CELLS;
  CKS(dalloc(hd, &hd->lab, n));
  CKS(dalloc(hd, &hd->comp, n));
  CKS(dalloc(hd, &hd->band, n));
  hd->tcap = (int)std::min<size_t>(n / 64 + 1024, (size_t)1 << 30);
  CKS(dalloc(hd, &hd->troots, (size_t)hd->tcap));
  CKS(dalloc(hd, &hd->cnt, nblk));
  CKS(dalloc(hd, &hd->dint, 4));
  CKS(dalloc(hd, &hd->roots, (size_t)DEFL_MAX));
  CKS(dalloc(hd, &hd->bflag, n));
  CKS(dalloc(hd, &hd->einv, (size_t)DEFL_MAX));
  CKS(dalloc(hd, &hd->coef, (size_t)DEFL_MAX));
  CKS(dalloc(hd, &hd->coef32, (size_t)DEFL_MAX));
  CKS(dalloc(hd, &hd->dscale, 4));
  CKS(dalloc(hd, &hd->acc_a, (size_t)DEFL_MAX * DEFL_REP * 2));
  CKS(dalloc(hd, &hd->acc_b, (size_t)DEFL_MAX * DEFL_REP * 2));
  CKS(dalloc(hd, &hd->acc_ztb, (size_t)DEFL_MAX * DEFL_REP * 2));
  CKS(dalloc(hd, &hd->dmax, 2));
  if (cudaMallocHost((void **)&hd->hint, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    hd->hint = nullptr;
    return MP_ERR_OOM;
  }
  CK(cudaStreamCreateWithFlags(&hd->cap, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&hd->cs, cudaStreamNonBlocking));
  for (cudaEvent_t &e : hd->xev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // coarse tail: the coarsest levels whose iterate, rhs and faces fit the
  // shared-memory budget of one block (coarsest level always included)
  for (int pass = 0; pass < 2; ++pass) {
    size_t elem = pass == 0 ? sizeof(double) : sizeof(float);
    size_t budget = pass == 0 ? TAIL_BUDGET64 : TAIL_BUDGET32;
    int start = (int)hd->L.size() - 1;
    const size_t arrays = hd->outflow ? 7 : 6;  // + the outflow diagonal
    size_t bytes = arrays * hd->L.back().n * elem;
    while (start > 0 && bytes + arrays * hd->L[start - 1].n * elem <= budget) {
      --start;
      bytes += arrays * hd->L[start].n * elem;
    }
    if (pass == 0) {
      hd->tail64 = start;
      hd->tail64_bytes = bytes;
    } else {
      hd->tail32 = start;
      hd->tail32_bytes = bytes;
    }
  }
  // fused FP32 sweep: levels above the one-CTA tail with nx a multiple of 8
  CKS(fused_setup(hd));
  CKS(ctail_setup(hd));
  CK(cudaFuncSetAttribute(k_inverse_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)((GJ_SMEM_MAX + 1) * GJ_SMEM_MAX * sizeof(double))));
  CK(cudaFuncSetAttribute(k_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)std::max<size_t>(hd->tail64_bytes, 1)));
  CK(cudaFuncSetAttribute(k_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)std::max<size_t>(hd->tail32_bytes, 1)));
  // the zero fills of dalloc run on the legacy default stream, which a
  // non-blocking caller stream does not wait for: finish them here
  CK(cudaDeviceSynchronize());
  return MP_OK;
}

// D v = At v - At Z E^-1 Z^T At v (the deflated operator) of FP64 v (device,
// hd->n), into out; v and out distinct handle scratch vectors
mp_status deflated_apply(mp_poisson *hd, double *v, double *out) {
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_APPLY64, 0, hd->n * 48.0, k_apply_dot<double>, zgrid(l0.d), kBlock, v, out, l0.bx,
         l0.by, l0.bz, l0.diag, (const double *)nullptr, l0.d, zper_of(l0.d), hd->partial);
  CKS(launch_ok());
  CKS((defl_coef<double, double>(hd, v, l0.bx, l0.by, l0.bz, false)));
  return defl_sub<double, double>(hd, out, l0.bx, l0.by, l0.bz);
}

mp_status dot64(mp_poisson *hd, const double *a, const double *b, double *out) {
  LAUNCH(hd, K_DOT64, 0, hd->n * 16.0, k_dot<double>, VEC_BLOCKS, VEC_THREADS, a, b, hd->n,
         hd->partial);
  CKS(reduce(hd, VEC_BLOCKS, OP_STORE, S_TMP));
  CKS(read_scalars(hd));
  *out = hd->scal_h[S_TMP];
  return MP_OK;
}

}  // namespace

extern "C" {

void mp_opts_default(mp_opts *o) {
  if (!o) return;
  o->precision = 0;
  o->method = 0;
  o->initial_guess = 0;
  o->max_iters = 200;
  o->nu1 = 2;
  o->nu2 = 2;
  o->nu_growth = 2;
  o->nu_max = 12;
  o->inner_rtol = 3e-3;
  o->inner_max = 12;
  o->net_check = 0;
  o->deflate = 1;
  o->smoother = 1;
  o->label_limit = 8192;
  o->coarse_cluster = 1;
  o->stream = nullptr;
}

const char *mp_status_str(mp_status s) {
  switch (s) {
    case MP_OK: return "ok";
    case MP_ERR_INVALID_ARG: return "invalid argument";
    case MP_ERR_NOT_CONVERGED: return "not converged (max_iters reached)";
    case MP_ERR_DIVERGED: return "diverged (non-finite residual)";
    case MP_ERR_CUDA: return "CUDA error";
    case MP_ERR_OOM: return "out of memory";
    case MP_ERR_TIMEOUT: return "device wait timed out";
    case MP_ERR_NO_NET: return "learned initial guess requested but no network is set";
  }
  return "unknown status";
}

mp_status mp_poisson_setup(mp_handle *out, mp_grid g, double h, const mp_bc bc[3],
                           const double *phi_dev, double rho_l, double rho_g, double sigma,
                           const mp_opts *opts) {
  if (!out || !bc || !phi_dev) return MP_ERR_INVALID_ARG;
  *out = nullptr;
  mp_opts o;
  mp_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_opts(o)) return MP_ERR_INVALID_ARG;
  mp_poisson *hd = new (std::nothrow) mp_poisson();
  if (!hd) return MP_ERR_OOM;
  hd->opts = o;
  hd->st = (cudaStream_t)o.stream;
  mp_status s = create(hd, g, h, bc);
  if (s == MP_OK) {
    apply_nu(hd);
    s = geometry(hd, phi_dev, rho_l, rho_g, sigma);
  }
  if (s != MP_OK) {
    mp_poisson_destroy(hd);
    return s;
  }
  *out = hd;
  return MP_OK;
}

mp_status mp_poisson_set_geometry(mp_handle hd, const double *phi_dev, double rho_l, double rho_g,
                                  double sigma) {
  if (!hd) return MP_ERR_INVALID_ARG;
  return geometry(hd, phi_dev, rho_l, rho_g, sigma);
}

mp_status mp_poisson_deflated_energy(mp_handle hd, const float *q_dev, const float *t_dev,
                                     float *gq_dev, double *loss_out) {
  if (!hd || !q_dev || !t_dev || !loss_out) return MP_ERR_INVALID_ARG;
  if (!hd->opts.deflate || hd->defl_m <= 0 || hd->outflow) return MP_ERR_INVALID_ARG;
  if ((hd->diag_mode & 1) != 1) CKS(diag_fields(hd, 1));
  const size_t n = hd->n;
  CK(cudaMemsetAsync(hd->acc_a, 0, defl_acc_bytes(hd->defl_m), hd->st));
  CK(cudaMemsetAsync(hd->dmax, 0, sizeof(unsigned long long), hd->st));
  LAUNCH(hd, K_SCALE, 0, n * 12.0, k_f32_to_f64, VEC_BLOCKS, VEC_THREADS, q_dev, hd->dv, n);
  LAUNCH(hd, K_SCALE, 0, n * 12.0, k_f32_to_f64, VEC_BLOCKS, VEC_THREADS, t_dev, hd->r, n);
  CKS(launch_ok());
  CKS(deflated_apply(hd, hd->dv, hd->q));  // D q
  CKS(deflated_apply(hd, hd->r, hd->z));   // D t
  double qdq, qdt, tdt;
  CKS(dot64(hd, hd->dv, hd->q, &qdq));
  CKS(dot64(hd, hd->dv, hd->z, &qdt));
  CKS(dot64(hd, hd->r, hd->z, &tdt));
  if (!(qdq != 0.0 && tdt != 0.0) || !std::isfinite(qdq * tdt)) return MP_ERR_DIVERGED;
  *loss_out = 1.0 - qdt * qdt / (qdq * tdt);
  if (gq_dev) {
    const double a = -2.0 * qdt / (qdq * tdt), b = 2.0 * qdt * qdt / (qdq * qdq * tdt);
    LAUNCH(hd, K_SCALE, 0, n * 20.0, k_lincomb_f32, VEC_BLOCKS, VEC_THREADS, gq_dev, a,
           (const double *)hd->z, b, (const double *)hd->q, n);
    CKS(launch_ok());
  }
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_set_mass_flux(mp_handle hd, const double *mdot_dev) {
  if (!hd) return MP_ERR_INVALID_ARG;
  if (mdot_dev) {
    if (!hd->mdot) CKS(dalloc(hd, &hd->mdot, hd->n));
    CK(cudaMemcpyAsync(hd->mdot, mdot_dev, hd->n * sizeof(double), cudaMemcpyDeviceToDevice,
                       hd->st));
  }
  hd->has_mdot = mdot_dev != nullptr;
  // the jump source of the current geometry, with or without the flux jump
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_JUMP, 0, hd->n * (hd->has_mdot ? 56.0 : 48.0), k_jump, cell_grid(l0.d), kBlock,
         hd->phi, hd->kap, l0.bx, l0.by, l0.bz, hd->Jt, l0.d, hd->sigma, mdot_of(hd), hd->rho_l,
         hd->rho_g, hd->h);
  CKS(launch_ok());
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_set_opts(mp_handle hd, const mp_opts *opts) {
  if (!hd || !opts || !valid_opts(*opts)) return MP_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(hd->st));
  hd->opts = *opts;
  hd->st = (cudaStream_t)opts->stream;
  apply_nu(hd);
  destroy_graphs(hd);
  return MP_OK;
}

mp_status mp_poisson_solve(mp_handle hd, const double *rhs_dev, double *p_dev, double tol,
                           int *iterations, double *res_hist, int res_hist_cap,
                           int *res_hist_len) {
  if (!hd || !rhs_dev || !p_dev || !(tol > 0.0) || res_hist_cap < 0 ||
      (res_hist_cap > 0 && !res_hist))
    return MP_ERR_INVALID_ARG;
  std::vector<double> hist;
  CKS(assemble_rhs(hd, rhs_dev));
  mp_status s = solve_assembled(hd, p_dev, tol, &hist);
  if (iterations) *iterations = hd->stats.iterations;
  int m = std::min<int>((int)hist.size(), res_hist_cap);
  for (int i = 0; i < m; ++i) res_hist[i] = hist[i];
  if (res_hist_len) *res_hist_len = m;
  return s;
}

mp_status mp_poisson_project_step(mp_handle hd, double *ux, double *uy, double *uz, double *p,
                                  double tol, int *iterations) {
  if (!hd || !ux || !uy || !uz || !p || !(tol > 0.0)) return MP_ERR_INVALID_ARG;
  if (hd->outflow) return MP_ERR_INVALID_ARG;  // one boundary face slot per axis
  CKS(assemble_rhs_u(hd, ux, uy, uz));
  mp_status s = solve_assembled(hd, p, tol, nullptr);
  if (iterations) *iterations = hd->stats.iterations;
  if (s != MP_OK) return s;
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_PROJECT, 0, hd->n * 96.0, k_project, cell_grid(l0.d), kBlock, p, hd->phi, hd->kap,
         l0.bx, l0.by, l0.bz, ux, uy, uz, l0.d, 0, hd->sigma, 1.0 / hd->h, mdot_of(hd),
         hd->rho_l, hd->rho_g);
  CKS(launch_ok());
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

// The host-buffer step as a z-slab pipeline on two streams.  Uploads of u*
// run on the copy stream slab by slab; the assembly of a slab starts once it
// and the next slab (the z-high faces of its last plane) have arrived.  After
// the solve p is downloaded while the velocity correction runs slab by slab,
// each slab's three components downloaded as soon as it is corrected.  One
// cudaMemcpyAsync per array and slab.
mp_status project_step_host(mp_poisson *hd, double *ux_h, double *uy_h, double *uz_h, double *p_h,
                            double tol, int *iterations) {
  Level &l0 = hd->L[0];
  const Dims d = l0.d;
  const Slabs q = slabs_of(d);
  const size_t plane = (size_t)d.nx * d.ny;
  cudaEvent_t *in = hd->xev, *out = hd->xev + MAX_SLABS, ready = hd->xev[2 * MAX_SLABS],
              solved = hd->xev[2 * MAX_SLABS + 1];
  // the copy stream starts after the work already queued on st
  CK(cudaEventRecord(ready, hd->st));
  CK(cudaStreamWaitEvent(hd->cs, ready, 0));
  auto planes = [&](int s, size_t &k0, size_t &cnt) {
    k0 = (size_t)q.kb_lo(s) * q.zper;
    cnt = std::min((size_t)d.nz, (size_t)q.kb_hi(s) * q.zper) - k0;
  };
  for (int s = 0; s < q.count; ++s) {
    size_t k0, cnt;
    planes(s, k0, cnt);
    const size_t off = k0 * plane, bytes = cnt * plane * sizeof(double);
    CK(cudaMemcpyAsync(hd->ux + off, ux_h + off, bytes, cudaMemcpyHostToDevice, hd->cs));
    CK(cudaMemcpyAsync(hd->uy + off, uy_h + off, bytes, cudaMemcpyHostToDevice, hd->cs));
    CK(cudaMemcpyAsync(hd->uz + off, uz_h + off, bytes, cudaMemcpyHostToDevice, hd->cs));
    CK(cudaEventRecord(in[s], hd->cs));
  }
  if (hd->opts.initial_guess == 1) {
    CK(cudaMemcpyAsync(hd->pst, p_h, hd->n * sizeof(double), cudaMemcpyHostToDevice, hd->cs));
    CK(cudaEventRecord(solved, hd->cs));
  }
  const dim3 g = zgrid(d);
  for (int s = 0; s < q.count; ++s) {
    // the slab's last plane reads the z-high faces in the next slab (plane 0
    // after the last: the periodic image or the shared wall face)
    CK(cudaStreamWaitEvent(hd->st, in[s], 0));
    CK(cudaStreamWaitEvent(hd->st, in[s + 1 < q.count ? s + 1 : 0], 0));
    const int kb0 = q.kb_lo(s), nb = q.kb_hi(s) - kb0;
    size_t k0, cnt;
    planes(s, k0, cnt);
    LAUNCH(hd, K_ASSEMBLE_U, 0, cnt * plane * 40.0, k_assemble_u, dim3(g.x, g.y, nb), kBlock,
           (const double *)hd->ux, (const double *)hd->uy, (const double *)hd->uz,
           (const double *)hd->Jt, hd->b, d, q.zper, kb0, hd->h, hd->partial);
  }
  CKS(launch_ok());
  if (hd->opts.initial_guess == 1) CK(cudaStreamWaitEvent(hd->st, solved, 0));
  CKS(finish_rhs(hd, zblocks(d)));
  mp_status s = solve_assembled(hd, hd->pst, tol, nullptr);
  if (iterations) *iterations = hd->stats.iterations;
  if (s != MP_OK) return s;
  CK(cudaEventRecord(solved, hd->st));
  CK(cudaStreamWaitEvent(hd->cs, solved, 0));
  CK(cudaMemcpyAsync(p_h, hd->pst, hd->n * sizeof(double), cudaMemcpyDeviceToHost, hd->cs));
  for (int s2 = 0; s2 < q.count; ++s2) {
    size_t k0, cnt;
    planes(s2, k0, cnt);
    LAUNCH(hd, K_PROJECT, 0, cnt * plane * 96.0, k_project,
           dim3(cell_grid(d).x, cell_grid(d).y, (unsigned)cnt), kBlock, (const double *)hd->pst,
           (const double *)hd->phi, (const double *)hd->kap, (const double *)l0.bx,
           (const double *)l0.by, (const double *)l0.bz, hd->ux, hd->uy, hd->uz, d, (int)k0,
           hd->sigma, 1.0 / hd->h, mdot_of(hd), hd->rho_l, hd->rho_g);
    CKS(launch_ok());
    CK(cudaEventRecord(out[s2], hd->st));
    CK(cudaStreamWaitEvent(hd->cs, out[s2], 0));
    const size_t off = k0 * plane, bytes = cnt * plane * sizeof(double);
    CK(cudaMemcpyAsync(ux_h + off, hd->ux + off, bytes, cudaMemcpyDeviceToHost, hd->cs));
    CK(cudaMemcpyAsync(uy_h + off, hd->uy + off, bytes, cudaMemcpyDeviceToHost, hd->cs));
    CK(cudaMemcpyAsync(uz_h + off, hd->uz + off, bytes, cudaMemcpyDeviceToHost, hd->cs));
  }
  CK(cudaStreamSynchronize(hd->cs));
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_project_step_host(mp_handle hd, double *ux_h, double *uy_h, double *uz_h,
                                       double *p_h, double tol, int *iterations) {
  if (!hd || !ux_h || !uy_h || !uz_h || !p_h || !(tol > 0.0)) return MP_ERR_INVALID_ARG;
  if (hd->outflow) return MP_ERR_INVALID_ARG;  // one boundary face slot per axis
  const mp_status s = project_step_host(hd, ux_h, uy_h, uz_h, p_h, tol, iterations);
  // no copy may touch the caller's buffers after the call returns
  const cudaError_t e = cudaStreamSynchronize(hd->cs);
  if (s == MP_OK && e != cudaSuccess) return MP_ERR_CUDA;
  return s;
}

mp_status mp_poisson_apply(mp_handle hd, const double *x, double *y) {
  if (!hd || !x || !y) return MP_ERR_INVALID_ARG;
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_APPLY64, 0, hd->n * 48.0, k_apply_dot<double>, zgrid(l0.d), kBlock, x, y,
         l0.bx, l0.by, l0.bz, l0.diag, (const double *)nullptr, l0.d, zper_of(l0.d), hd->partial);
  LAUNCH(hd, K_SCALE, 0, hd->n * 16.0, k_scale, VEC_BLOCKS, VEC_THREADS, y, y, hd->n,
         1.0 / (hd->h * hd->h));
  CKS(launch_ok());
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_divergence(mp_handle hd, const double *ux, const double *uy,
                                const double *uz, double *dv) {
  if (!hd || !ux || !uy || !uz || !dv) return MP_ERR_INVALID_ARG;
  if (hd->outflow) return MP_ERR_INVALID_ARG;  // one boundary face slot per axis
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_DIV, 0, hd->n * 32.0, k_divergence, cell_grid(l0.d), kBlock, ux, uy, uz, dv, l0.d,
         hd->h);
  CKS(launch_ok());
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_rhs(mp_handle hd, const double *rhs, double *b) {
  if (!hd || !rhs || !b) return MP_ERR_INVALID_ARG;
  CKS(assemble_rhs(hd, rhs));
  LAUNCH(hd, K_SCALE, 0, hd->n * 16.0, k_scale, VEC_BLOCKS, VEC_THREADS, hd->b, b, hd->n,
         1.0 / (hd->h * hd->h));
  CKS(launch_ok());
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_project(mp_handle hd, const double *p, double *ux, double *uy, double *uz) {
  if (!hd || !p || !ux || !uy || !uz) return MP_ERR_INVALID_ARG;
  if (hd->outflow) return MP_ERR_INVALID_ARG;  // one boundary face slot per axis
  Level &l0 = hd->L[0];
  LAUNCH(hd, K_PROJECT, 0, hd->n * 96.0, k_project, cell_grid(l0.d), kBlock, p, hd->phi, hd->kap,
         l0.bx, l0.by, l0.bz, ux, uy, uz, l0.d, 0, hd->sigma, 1.0 / hd->h, mdot_of(hd),
         hd->rho_l, hd->rho_g);
  CKS(launch_ok());
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_get_fields(mp_handle hd, double *kappa, double *bx, double *by, double *bz,
                                double *J) {
  if (!hd) return MP_ERR_INVALID_ARG;
  Level &l0 = hd->L[0];
  size_t bytes = hd->n * sizeof(double);
  if (kappa) CK(cudaMemcpyAsync(kappa, hd->kap, bytes, cudaMemcpyDeviceToDevice, hd->st));
  if (bx) CK(cudaMemcpyAsync(bx, l0.bx, bytes, cudaMemcpyDeviceToDevice, hd->st));
  if (by) CK(cudaMemcpyAsync(by, l0.by, bytes, cudaMemcpyDeviceToDevice, hd->st));
  if (bz) CK(cudaMemcpyAsync(bz, l0.bz, bytes, cudaMemcpyDeviceToDevice, hd->st));
  if (J) {
    LAUNCH(hd, K_SCALE, 0, hd->n * 16.0, k_scale, VEC_BLOCKS, VEC_THREADS, hd->Jt, J, hd->n,
           1.0 / (hd->h * hd->h));
    CKS(launch_ok());
  }
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  return MP_OK;
}

mp_status mp_poisson_set_profiling(mp_handle hd, int enable) {
  if (!hd) return MP_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  if (enable && hd->events.empty()) {
    hd->events.resize(EVENT_POOL);
    for (auto &e : hd->events) CK(cudaEventCreate(&e));
  }
  hd->prof_on = enable ? 1 : 0;
  for (auto &row : hd->prof)
    for (auto &e : row) e = ProfEntry{};
  return MP_OK;
}

mp_status mp_poisson_get_profile(mp_handle hd, mp_kernel_prof *out, int cap, int *count) {
  if (!hd || cap < 0 || (cap > 0 && !out)) return MP_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(hd->st));
  prof_resolve(hd);
  int m = 0;
  for (int k = 0; k < K_COUNT; ++k)
    for (int l = 0; l < MAX_LEVELS; ++l) {
      const ProfEntry &e = hd->prof[k][l];
      if (e.launches == 0) continue;
      if (m < cap) {
        mp_kernel_prof &o = out[m];
        std::snprintf(o.name, sizeof(o.name), "%s", kKernelNames[k]);
        o.level = l;
        o.cells = l < (int)hd->L.size() ? (long long)hd->L[l].n : 0;
        o.launches = e.launches;
        o.total_ms = e.ms;
        o.alg_bytes = e.bytes;
      }
      ++m;
    }
  if (count) *count = m;
  return MP_OK;
}

mp_status mp_poisson_set_net(mp_handle hd, mp_net_handle net) {
  if (!hd) return MP_ERR_INVALID_ARG;
  if (net) {
    int nx = 0, ny = 0, nz = 0;
    CKS(mp_net_dims(net, &nx, &ny, &nz));
    if (nx == hd->g.nx && ny == hd->g.ny && nz == hd->g.nz)
      hd->net_factor = 1;
    else if (2 * nx == hd->g.nx && 2 * ny == hd->g.ny && 2 * nz == hd->g.nz)
      hd->net_factor = 2;
    else
      return MP_ERR_INVALID_ARG;
  }
  hd->net = net;
  return MP_OK;
}

mp_status mp_poisson_get_components(mp_handle hd, int *comp_dev, int *m) {
  if (!hd) return MP_ERR_INVALID_ARG;
  if (comp_dev) {
    CK(cudaMemcpyAsync(comp_dev, hd->comp, hd->n * sizeof(int), cudaMemcpyDeviceToDevice, hd->st));
    CK(cudaStreamSynchronize(hd->st));
  }
  if (m) *m = hd->defl_m;
  return MP_OK;
}

mp_status mp_poisson_get_stats(mp_handle hd, mp_stats *st) {
  if (!hd || !st) return MP_ERR_INVALID_ARG;
  *st = hd->stats;
  return MP_OK;
}

void mp_poisson_destroy(mp_handle hd) {
  if (!hd) return;
  cudaStreamSynchronize(hd->st);
  for (void *p : hd->allocs) cudaFree(p);
  for (cudaEvent_t e : hd->events) cudaEventDestroy(e);
  destroy_graphs(hd);
  if (hd->cap) cudaStreamDestroy(hd->cap);
  if (hd->cs) {
    cudaStreamSynchronize(hd->cs);
    cudaStreamDestroy(hd->cs);
  }
  for (cudaEvent_t e : hd->xev)
    if (e) cudaEventDestroy(e);
  if (hd->scal_h) cudaFreeHost(hd->scal_h);
  if (hd->hint) cudaFreeHost(hd->hint);
  delete hd;
}

}  // extern "C"
