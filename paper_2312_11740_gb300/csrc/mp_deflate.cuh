// Deflation of the MG-preconditioned CG by the gas components (bubbles).
//
// At density ratio 1000 the slowest error components of the V-cycle are the
// pressure levels of the individual gas regions: inside a bubble the
// coefficient is 1000x that of the liquid, the level is set only through the
// thin interface layer, and after two or three coarsenings a small bubble is
// no longer resolved by the coarse grids.  CG is therefore deflated by the
// indicator vectors z_j of the connected gas components (Tang & Vuik's
// deflated PCG for bubbly flows): with Z = [z_1 .. z_m], E = Z^T A Z and
// P = I - A Z E^-1 Z^T, CG starts from the residual P r0, projects every
// preconditioned residual, z <- P^T z (the A-DEF2 form of Tang, Nabben, Vuik
// and Erlangga, which tolerates rounding), and the solution is
// x + Z E^-1 Z^T (b - A x).  Components never share a face, so E is diagonal
// (E_jj = -sum of the face coefficients on component j's boundary), and for
// any v the products Z^T A v and A Z c are nonzero only on the band of cells
// with a face to another component (or to liquid): the per-iteration work is a
// few passes over that band and one fused pass over the grid.
//
// Components come from a union-find labelling of the gas cells (lowest cell
// index as root); ids follow the roots' cell order, and every sum over cells
// uses fixed-point int64 atomics, so results are bitwise reproducible.
#pragma once

namespace mp {

constexpr int DEFL_MAX = 4096;          // components handled (more: deflation off)
constexpr int DEFL_REP = 16;            // replicas of each accumulator (atomic contention)
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_TILE = 8 * SCAN_THREADS;  // counts scanned per pass (in shared memory)
constexpr int BAND_THREADS = 256;
constexpr int BAND_ROUNDS = 8;
constexpr int BAND_CELLS = BAND_THREADS * BAND_ROUNDS;  // cells per compaction block

// (i, j, k) of cell c in 32-bit arithmetic (deflation requires n < 2^31)
__device__ __forceinline__ void cell_ijk(const Dims &d, size_t c, int &i, int &j, int &k) {
  const unsigned u = (unsigned)c, t = u / (unsigned)d.nx;
  i = (int)(u - t * (unsigned)d.nx);
  j = (int)(t % (unsigned)d.ny);
  k = (int)(t / (unsigned)d.ny);
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// root of x.  Labels only decrease (lab[x] <= x always), so walks end at a
// root; path halving (lab[x] <- lab[lab[x]], by atomicMin) keeps them short.
// Every labelling loop stops after `limit` rounds (mp_opts.label_limit) and
// raises *err, which turns deflation off for the geometry.
__device__ __forceinline__ int ccl_find(int *lab, int x, int *err, int limit) {
  for (int it = 0; it < limit; ++it) {
    const int p = ld_volatile(lab + x);
    if (p == x) return x;
    const int g = ld_volatile(lab + p);
    if (g < p) atomicMin(lab + x, g);
    x = p;
  }
  atomicExch(err, 1);
  return x;
}

// union of the components of a and b: the larger root is hooked under the
// smaller with atomicMin, retried on the new root if another thread got there
__device__ void ccl_unite(int *lab, int a, int b, int *err, int limit) {
  for (int it = 0; it < limit; ++it) {
    a = ccl_find(lab, a, err, limit);
    b = ccl_find(lab, b, err, limit);
    if (a == b) return;
    if (a < b) {
      const int old = atomicMin(lab + b, a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(lab + a, b);
      if (old == a) return;
      a = old;
    }
  }
  atomicExch(err, 1);
}

// Two-pass labelling.  Pass 1 (k_ccl_tile): a 32 x 8 x 8 tile of cells is
// labelled in shared memory (union-find on local indices, which order the
// cells as their global indices do), and every gas cell gets the global index
// of its local root -- the smallest cell of its local component, so labels
// still only decrease.  Pass 2 (k_ccl_faces): only the cells on a tile's high
// faces unite, globally, with their neighbour across the face (periodic axes
// wrap), their finds one hop long.  The global unions drop from three per gas
// cell to about one per four cells, which matters when one component fills
// most of the grid (the gas above a liquid pool).
constexpr int CT_X = 32, CT_Y = 8, CT_Z = 8, CT_CELLS = CT_X * CT_Y * CT_Z, CT_THREADS = 512;

__device__ __forceinline__ int ct_find(int *L, int x, int *err, int limit) {
  const volatile int *V = L;  // other threads hook and halve concurrently
  for (int it = 0; it < limit; ++it) {
    const int p = V[x];
    if (p == x) return x;
    const int g = V[p];
    if (g < p) atomicMin(L + x, g);
    x = p;
  }
  atomicExch(err, 1);
  return x;
}
__device__ void ct_unite(int *L, int a, int b, int *err, int limit) {
  for (int it = 0; it < limit; ++it) {
    a = ct_find(L, a, err, limit);
    b = ct_find(L, b, err, limit);
    if (a == b) return;
    if (a < b) {
      const int old = atomicMin(L + b, a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(L + a, b);
      if (old == a) return;
      a = old;
    }
  }
  atomicExch(err, 1);
}

// (troots: every tile root's cell index, the first cap of them; *ntroots
// counts all)
__global__ void __launch_bounds__(CT_THREADS) k_ccl_tile(const double *__restrict__ phi,
                                                         int *__restrict__ lab, Dims d, int *err,
                                                         int limit, int *__restrict__ troots,
                                                         int *ntroots, int cap) {
  __shared__ int L[CT_CELLS];
  const int tx = blockIdx.x * CT_X, ty = blockIdx.y * CT_Y, tz = blockIdx.z * CT_Z;
  // local index li = x + CT_X (y + CT_Y z); cells outside the grid are liquid
  int mine_gas = 1, mine_liq = 1;
  for (int li = threadIdx.x; li < CT_CELLS; li += CT_THREADS) {
    const int x = tx + li % CT_X, y = ty + (li / CT_X) % CT_Y, z = tz + li / (CT_X * CT_Y);
    const bool in = x < d.nx && y < d.ny && z < d.nz;
    const bool g = in && gas(phi[at(d, x, y, z)]);
    L[li] = g ? li : -1;
    mine_gas &= g ? 1 : 0;
    mine_liq &= g ? 0 : 1;
  }
  // a tile that is all gas (one component, rooted at its first cell) or all
  // liquid needs no unions (most tiles of a pool or a large bubble)
  const int all_gas = __syncthreads_and(mine_gas), all_liq = __syncthreads_and(mine_liq);
  if (all_gas || all_liq) {
    const int root = all_gas ? (int)at(d, tx, ty, tz) : -1;
    for (int li = threadIdx.x; li < CT_CELLS; li += CT_THREADS) {
      const int x = tx + li % CT_X, y = ty + (li / CT_X) % CT_Y, z = tz + li / (CT_X * CT_Y);
      if (x < d.nx && y < d.ny && z < d.nz) lab[at(d, x, y, z)] = root;
    }
    if (all_gas && threadIdx.x == 0) {
      const int q = atomicAdd(ntroots, 1);
      if (q < cap) troots[q] = root;
    }
    return;
  }
  for (int li = threadIdx.x; li < CT_CELLS; li += CT_THREADS) {
    if (L[li] < 0) continue;
    const int lx = li % CT_X, ly = (li / CT_X) % CT_Y, lz = li / (CT_X * CT_Y);
    if (lx + 1 < CT_X && L[li + 1] >= 0) ct_unite(L, li, li + 1, err, limit);
    if (ly + 1 < CT_Y && L[li + CT_X] >= 0) ct_unite(L, li, li + CT_X, err, limit);
    if (lz + 1 < CT_Z && L[li + CT_X * CT_Y] >= 0) ct_unite(L, li, li + CT_X * CT_Y, err, limit);
  }
  __syncthreads();
  for (int li = threadIdx.x; li < CT_CELLS; li += CT_THREADS) {
    const int x = tx + li % CT_X, y = ty + (li / CT_X) % CT_Y, z = tz + li / (CT_X * CT_Y);
    if (x >= d.nx || y >= d.ny || z >= d.nz) continue;
    int v = -1;
    if (L[li] >= 0) {
      const int r = ct_find(L, li, err, limit);
      v = (int)at(d, tx + r % CT_X, ty + (r / CT_X) % CT_Y, tz + r / (CT_X * CT_Y));
      if (r == li) {
        const int q = atomicAdd(ntroots, 1);
        if (q < cap) troots[q] = v;
      }
    }
    lab[at(d, x, y, z)] = v;
  }
}

// unite the gas cells on the high faces of every tile with their gas
// neighbour across the face (wrapping on periodic axes only)
__global__ void __launch_bounds__(CT_THREADS) k_ccl_faces(int *lab, Dims d, int per, int *err,
                                                          int limit) {
  const int tx = blockIdx.x * CT_X, ty = blockIdx.y * CT_Y, tz = blockIdx.z * CT_Z;
  const int xe = min(CT_X, d.nx - tx), ye = min(CT_Y, d.ny - ty), ze = min(CT_Z, d.nz - tz);
  // the face cells of the tile: x = xe-1 (ye * ze), y = ye-1 (xe * ze), z = ze-1 (xe * ye)
  const int nfx = ye * ze, nfy = xe * ze, nfz = xe * ye;
  for (int e = threadIdx.x; e < nfx + nfy + nfz; e += CT_THREADS) {
    int x, y, z, dir;
    if (e < nfx) {
      x = xe - 1; y = e % ye; z = e / ye; dir = 0;
    } else if (e < nfx + nfy) {
      const int f = e - nfx;
      y = ye - 1; x = f % xe; z = f / xe; dir = 1;
    } else {
      const int f = e - nfx - nfy;
      z = ze - 1; x = f % xe; y = f / xe; dir = 2;
    }
    x += tx;
    y += ty;
    z += tz;
    const int c = (int)at(d, x, y, z);
    if (ld_volatile(lab + c) < 0) continue;
    int nb = -1;
    if (dir == 0 && (x + 1 < d.nx || (per & 1))) nb = (int)at(d, whi(x, d.nx), y, z);
    if (dir == 1 && (y + 1 < d.ny || (per & 2))) nb = (int)at(d, x, whi(y, d.ny), z);
    if (dir == 2 && (z + 1 < d.nz || (per & 4))) nb = (int)at(d, x, y, whi(z, d.nz));
    if (nb >= 0 && ld_volatile(lab + nb) >= 0) ccl_unite(lab, c, nb, err, limit);
  }
}

// lab[c] <- root of c for every gas cell; every root appends its index to
// roots (first DEFL_MAX of them; *nroots counts all)
//
// Two passes when every tile root is listed (*ntroots <= cap): the tile roots
// find their roots first (k_ccl_flatten_roots), then every cell takes one
// hop -- after the tile pass each cell points at its tile root, and the
// unions and path halving only ever re-point a cell at another tile root, so
// lab[lab[c]] is c's root.  Otherwise every cell walks to its root.
__global__ void k_ccl_flatten_roots(int *lab, const int *__restrict__ troots,
                                    const int *__restrict__ ntroots, int cap, int *err,
                                    int *roots, int *nroots, int limit) {
  const int nt = *ntroots;
  if (nt > cap) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    const int t = troots[q];
    const int r = ccl_find(lab, t, err, limit);
    lab[t] = r;
    if (r == t) {
      const int w = atomicAdd(nroots, 1);
      if (w < DEFL_MAX) roots[w] = r;
    }
  }
}

__global__ void k_ccl_flatten(int *lab, size_t n, int *err, int *roots, int *nroots, int limit,
                              const int *__restrict__ ntroots, int cap) {
  if (*ntroots <= cap) {
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
      const int p = lab[c];
      if (p >= 0) lab[c] = lab[p];
    }
    return;
  }
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    if (lab[c] < 0) continue;
    const int r = ccl_find(lab, (int)c, err, limit);
    lab[c] = r;
    if (r == (int)c) {
      const int q = atomicAdd(nroots, 1);
      if (q < DEFL_MAX) roots[q] = r;
    }
  }
}

// comp[root] = rank of the root's cell index among all roots (ids follow the
// roots' cell order whatever order the roots were appended in).  One block.
__global__ void k_rank_roots(const int *__restrict__ roots, const int *__restrict__ nroots,
                             int *__restrict__ comp) {
  __shared__ int sr[DEFL_MAX];
  const int m = *nroots;
  if (m > DEFL_MAX) return;  // deflation is off for this geometry
  for (int q = threadIdx.x; q < m; q += blockDim.x) sr[q] = roots[q];
  __syncthreads();
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const int v = sr[q];
    int rank = 0;
    for (int e = 0; e < m; ++e) rank += sr[e] < v;
    comp[v] = rank;
  }
}

// comp[c] = id of c's root (roots already hold their id), -1 for liquid
__global__ void k_comp_from_roots(const int *__restrict__ lab, int *comp, size_t n) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const int r = lab[c];
    comp[c] = r < 0 ? -1 : comp[r];
  }
}

// ------------------------------------------ ordered band compaction (scan)
// band cell: a face neighbour (wrapped as in the stencils) has another id
__device__ __forceinline__ bool band_flag(const int *__restrict__ comp, const Dims &d, size_t c) {
  int i, j, k;
  cell_ijk(d, c, i, j, k);
  const int m = comp[c];
  return comp[at(d, wlo(i, d.nx), j, k)] != m || comp[at(d, whi(i, d.nx), j, k)] != m ||
         comp[at(d, i, wlo(j, d.ny), k)] != m || comp[at(d, i, whi(j, d.ny), k)] != m ||
         comp[at(d, i, j, wlo(k, d.nz))] != m || comp[at(d, i, j, whi(k, d.nz))] != m;
}

// number of band cells in each block of BAND_CELLS consecutive cells; the
// per-cell flags are kept (one byte each) for k_band_assign
__global__ void __launch_bounds__(BAND_THREADS) k_band_count(const int *__restrict__ comp, Dims d,
                                                             size_t n, int *__restrict__ cnt,
                                                             unsigned char *__restrict__ flag) {
  const size_t base = (size_t)blockIdx.x * BAND_CELLS;
  int total = 0;
#pragma unroll
  for (int r = 0; r < BAND_ROUNDS; ++r) {
    const size_t c = base + (size_t)r * BAND_THREADS + threadIdx.x;
    const bool f = c < n && band_flag(comp, d, c);
    if (c < n) flag[c] = f ? 1 : 0;
    total += __syncthreads_count(f);
  }
  if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// exclusive scan of nb counts in place (one block of SCAN_THREADS), total -> *total.
// Each pass stages SCAN_TILE counts in shared memory (coalesced), every thread
// sums 8 consecutive ones, and a two-level warp-shuffle scan gives the offsets.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_counts(int *cnt, int nb, int *total) {
  __shared__ int tile[SCAN_TILE];
  __shared__ int wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int carry = 0;
  for (int t0 = 0; t0 < nb; t0 += SCAN_TILE) {
    for (int q = t; q < SCAN_TILE; q += SCAN_THREADS) tile[q] = t0 + q < nb ? cnt[t0 + q] : 0;
    __syncthreads();
    int s = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) s += tile[t * 8 + e];
    int incl = s;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int v = wsum[lane];
      int wi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += u;
      }
      wsum[lane] = wi;  // inclusive over warps
    }
    __syncthreads();
    const int tile_total = wsum[31];
    int run = carry + (w > 0 ? wsum[w - 1] : 0) + incl - s;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int v = tile[t * 8 + e];
      tile[t * 8 + e] = run;
      run += v;
    }
    __syncthreads();
    for (int q = t; q < SCAN_TILE; q += SCAN_THREADS)
      if (t0 + q < nb) cnt[t0 + q] = tile[q];
    carry += tile_total;
    __syncthreads();
  }
  if (t == 0) *total = carry;
}

// band[id] = c for the band cells, in cell order (off: the scanned counts)
__global__ void __launch_bounds__(BAND_THREADS) k_band_assign(const unsigned char *__restrict__ flag,
                                                              size_t n, const int *__restrict__ off,
                                                              int *__restrict__ band) {
  __shared__ int wcount[BAND_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t base = (size_t)blockIdx.x * BAND_CELLS;
  int run = off[blockIdx.x];
  for (int r = 0; r < BAND_ROUNDS; ++r) {
    const size_t c = base + (size_t)r * BAND_THREADS + threadIdx.x;
    const bool f = c < n && flag[c] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcount[w] = __popc(bal);
    __syncthreads();
    int wb = run, tot = 0;
#pragma unroll
    for (int q = 0; q < BAND_THREADS / 32; ++q) {
      if (q < w) wb += wcount[q];
      tot += wcount[q];
    }
    if (f) band[wb + __popc(bal & ((1u << lane) - 1u))] = (int)c;
    run += tot;
    __syncthreads();
  }
}

// ----------------------------------------- fixed-point deterministic sums
// A sum is accumulated as v * scale in two int64 words per replica: the
// nearest integer (hi) and the remaining fraction in units of 2^-28 (lo).
// The caller's scale bounds |sum of v * scale| by 2^60, so hi cannot
// overflow; the fraction word extends the resolution to 2^-88 of that bound,
// which keeps the sums exact to FP64 rounding even when the bound is far above
// the sum (a whole-grid bound for a small bubble).  Integer addition is
// associative, so every sum is bitwise reproducible.
constexpr double FX_LO = 268435456.0;  // 2^28

__device__ __forceinline__ unsigned long long *fx_slot(unsigned long long *acc, int j, int rep) {
  return acc + ((size_t)j * DEFL_REP + rep) * 2;
}
__device__ __forceinline__ void fx_add(unsigned long long *acc, int j, double v, double scale) {
  const double y = v * scale;
  const double yh = rint(y);
  const long long hi = (long long)yh;
  const long long lo = llrint((y - yh) * FX_LO);  // y - yh is exact
  unsigned long long *a = fx_slot(acc, j, blockIdx.x % DEFL_REP);
  if (hi != 0) atomicAdd(a, (unsigned long long)hi);
  if (lo != 0) atomicAdd(a + 1, (unsigned long long)lo);
}
// the sum of component j (clear: zero its words after reading)
__device__ __forceinline__ double fx_value(unsigned long long *acc, int j, double scale,
                                           bool clear) {
  long long hi = 0, lo = 0;
#pragma unroll
  for (int q = 0; q < DEFL_REP; ++q) {
    unsigned long long *a = fx_slot(acc, j, q);
    hi += (long long)a[0];
    lo += (long long)a[1];
    if (clear) a[0] = a[1] = 0ull;
  }
  return ((double)hi + (double)lo / FX_LO) / scale;
}

// (A z_j)_c of band cell c for every component j it touches (A = sum_f
// beta_f (x_nb - x_c)): slot f < 6 holds +beta_f for the component k_f of a
// face neighbour outside comp(c); slot 6 holds, for c in component m, minus
// the sum of its faces to other ids.  k = -1 marks an empty slot.
template <typename F>
__device__ __forceinline__ void band_row(const F *__restrict__ bx, const F *__restrict__ by,
                                         const F *__restrict__ bz, const int *__restrict__ comp,
                                         const Dims &d, size_t c, int ks[7], double ws[7]) {
  int i, j, k;
  cell_ijk(d, c, i, j, k);
  const int m = comp[c];
  const size_t nb[6] = {at(d, wlo(i, d.nx), j, k), at(d, whi(i, d.nx), j, k),
                        at(d, i, wlo(j, d.ny), k), at(d, i, whi(j, d.ny), k),
                        at(d, i, j, wlo(k, d.nz)), at(d, i, j, whi(k, d.nz))};
  const double w[6] = {(double)bx[c], (double)bx[nb[1]], (double)by[c],
                       (double)by[nb[3]], (double)bz[c], (double)bz[nb[5]]};
  double self = 0.0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int mk = comp[nb[f]];
    const bool cross = mk != m && w[f] != 0.0;
    if (cross && m >= 0) self += w[f];
    ks[f] = cross && mk >= 0 ? mk : -1;
    ws[f] = w[f];
  }
  ks[6] = m >= 0 && self != 0.0 ? m : -1;
  ws[6] = -self;
}

// A warp's running FP64 sum for one component, carried across grid-stride
// chunks and added to the fixed-point accumulator when the component changes
// (and by flush at the end): one atomic add per warp and component run.
// Every lane holds the same state.
struct FxCarry {
  int cur = -1;
  double run = 0.0;
  __device__ __forceinline__ void add(unsigned long long *acc, int m, double s, double scale) {
    if (m == cur) {
      run += s;
      return;
    }
    flush(acc, scale);
    cur = m;
    run = s;
  }
  __device__ __forceinline__ void flush(unsigned long long *acc, double scale) {
    if (cur >= 0 && (threadIdx.x & 31) == 0 && run != 0.0) fx_add(acc, cur, run, scale);
    cur = -1;
    run = 0.0;
  }
};

// Warp-aggregated fixed-point add of the (ks[f], vals[f]) pairs of every lane:
// the contributions to the warp's leading component (the first one met in
// lane order) are summed across the warp in a fixed shuffle tree and carried
// in `carry`; the others are added per lane.  Called by all 32 lanes.
__device__ __forceinline__ void fx_add_warp(unsigned long long *acc, const int ks[7],
                                            const double vals[7], double scale, FxCarry &carry) {
  int mine = -1;
#pragma unroll
  for (int f = 0; f < 7; ++f)
    if (mine < 0 && ks[f] >= 0) mine = ks[f];
  const unsigned has = __ballot_sync(0xffffffffu, mine >= 0);
  if (has == 0u) return;
  const int mm = __shfl_sync(0xffffffffu, mine, __ffs(has) - 1);
  double s = 0.0;
  bool other = false;
#pragma unroll
  for (int f = 0; f < 7; ++f) {
    if (ks[f] == mm)
      s += vals[f];
    else if (ks[f] >= 0)
      other = true;
  }
  s = warp_sum(s);
  carry.add(acc, mm, s, scale);
  if (other) {
#pragma unroll
    for (int f = 0; f < 7; ++f)
      if (ks[f] >= 0 && ks[f] != mm) fx_add(acc, ks[f], vals[f], scale);
  }
}

// E_jj = z_j^T A z_j over the band (fixed point, scale)
template <typename F>
__global__ void k_defl_E(const int *__restrict__ band, int nband, const int *__restrict__ comp,
                         const F *__restrict__ bx, const F *__restrict__ by,
                         const F *__restrict__ bz, Dims d, unsigned long long *acc, double scale) {
  const int stride = gridDim.x * blockDim.x;
  FxCarry carry;
  for (int e0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < nband; e0 += stride) {
    const int e = e0 + (threadIdx.x & 31);
    int ks[7];
    double ws[7];
#pragma unroll
    for (int f = 0; f < 7; ++f) ks[f] = -1, ws[f] = 0.0;
    if (e < nband) band_row(bx, by, bz, comp, d, (size_t)band[e], ks, ws);
#pragma unroll
    for (int f = 0; f < 6; ++f) ks[f] = -1;  // only the diagonal term z_j^T A z_j
    fx_add_warp(acc, ks, ws, scale, carry);
  }
  carry.flush(acc, scale);
}

// max |v| over the band (as the ordered bits of a non-negative double)
template <typename T>
__global__ void k_defl_maxabs(const int *__restrict__ band, int nband, const T *__restrict__ v,
                              unsigned long long *mx) {
  double m = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nband; e += gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)v[band[e]]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

// sums[j] += sum over the band of (A z_j)_c v_c  ( = (A Z)^T v ), scale from the
// band maximum of |v| (6 faces of at most beta_max each)
template <typename T, typename F>
__global__ void k_defl_azt(const int *__restrict__ band, int nband, const int *__restrict__ comp,
                           const F *__restrict__ bx, const F *__restrict__ by,
                           const F *__restrict__ bz, Dims d, const T *__restrict__ v,
                           const unsigned long long *__restrict__ mx, double beta_max,
                           unsigned long long *acc, double *scale_out) {
  griddep_wait();
  const double vmax = __longlong_as_double((long long)*mx);
  const double bound = vmax * 6.0 * beta_max * (double)nband;
  const double scale = bound > 0.0 ? ldexp(1.0, 60) / bound : 1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = scale;
  const int stride = gridDim.x * blockDim.x;
  FxCarry carry;
  for (int e0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < nband; e0 += stride) {
    const int e = e0 + (threadIdx.x & 31);
    int ks[7];
    double ws[7];
#pragma unroll
    for (int f = 0; f < 7; ++f) ks[f] = -1, ws[f] = 0.0;
    if (e < nband) {
      const size_t c = (size_t)band[e];
      band_row(bx, by, bz, comp, d, c, ks, ws);
      const double vc = (double)v[c];
#pragma unroll
      for (int f = 0; f < 7; ++f) ws[f] *= vc;
    }
    fx_add_warp(acc, ks, ws, scale, carry);
  }
  carry.flush(acc, scale);
}

// sums[j] += sum of v over all cells of component j (|sum| bounded by the caller's scale).
// A warp whose 32 cells hold one component sums them in a fixed shuffle tree
// and carries that sum in FP64 across its grid-stride chunks while the
// component stays the same, adding it to the fixed-point accumulator only
// when the component changes and at the end: a large component (the gas
// above a liquid pool) costs one atomic add per warp instead of one per 32
// cells.  Fixed launch shape, fixed order: bitwise reproducible.
template <typename T>
__global__ void k_defl_zt(const int *__restrict__ comp, const T *__restrict__ v, size_t n,
                          unsigned long long *acc, double scale) {
  FxCarry carry;
  for (size_t c0 = blockIdx.x * (size_t)blockDim.x; c0 < n; c0 += (size_t)gridDim.x * blockDim.x) {
    const size_t c = c0 + threadIdx.x;
    const int m = c < n ? comp[c] : -1;
    const double val = m >= 0 ? (double)v[c] : 0.0;
    const unsigned gasl = __ballot_sync(0xffffffffu, m >= 0);
    if (gasl == 0u) continue;
    const int mm = __shfl_sync(0xffffffffu, m, __ffs(gasl) - 1);
    if (__all_sync(0xffffffffu, m < 0 || m == mm)) {
      carry.add(acc, mm, warp_sum(val), scale);
    } else if (m >= 0) {
      fx_add(acc, m, val, scale);
    }
  }
  carry.flush(acc, scale);
}

// c_j = E_jj^-1 (s_j - t_j): s from the sum sa (scale *scale_a, or fixed_scale_a
// when scale_a is null), t from the sum sb (scale *scale_b), either may be
// absent.  The per-projection sums (sb, or sa when clear_a) and the band
// maximum mx are zeroed for the next projection.
__global__ void k_defl_coef(int m, unsigned long long *sa, const double *scale_a,
                            double fixed_scale_a, int clear_a, unsigned long long *sb,
                            const double *scale_b, const double *__restrict__ einv,
                            double *__restrict__ coef, float *__restrict__ coef32,
                            unsigned long long *mx) {
  griddep_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) *mx = 0ull;
  if (j >= m) return;
  double s = 0.0;
  if (sa) s = fx_value(sa, j, scale_a ? *scale_a : fixed_scale_a, clear_a != 0);
  if (sb) s -= fx_value(sb, j, *scale_b, true);
  coef[j] = einv[j] * s;
  coef32[j] = (float)coef[j];
}

// (A w)_c of band cell c for w = coef[comp] (0 in liquid)
template <typename F>
__device__ __forceinline__ double band_aw(const F *__restrict__ bx, const F *__restrict__ by,
                                          const F *__restrict__ bz, const int *__restrict__ comp,
                                          const Dims &d, size_t c, int i, int j, int k,
                                          const double *__restrict__ coef) {
  const int m = comp[c];
  const double wc = m >= 0 ? coef[m] : 0.0;
  const size_t nb[6] = {at(d, wlo(i, d.nx), j, k), at(d, whi(i, d.nx), j, k),
                        at(d, i, wlo(j, d.ny), k), at(d, i, whi(j, d.ny), k),
                        at(d, i, j, wlo(k, d.nz)), at(d, i, j, whi(k, d.nz))};
  const double w[6] = {(double)bx[c], (double)bx[nb[1]], (double)by[c],
                       (double)by[nb[3]], (double)bz[c], (double)bz[nb[5]]};
  double aw = 0.0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int mk = comp[nb[f]];
    const double wn = mk >= 0 ? coef[mk] : 0.0;
    aw += w[f] * (wn - wc);
  }
  return aw;
}

// v_c -= (A w)_c on the band, w = coef[comp] (0 in liquid)
template <typename T, typename F>
__global__ void k_defl_sub_aw(const int *__restrict__ band, int nband, const int *__restrict__ comp,
                              const F *__restrict__ bx, const F *__restrict__ by,
                              const F *__restrict__ bz, Dims d, const double *__restrict__ coef,
                              T *__restrict__ v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nband; e += gridDim.x * blockDim.x) {
    const size_t c = (size_t)band[e];
    int i, j, k;
    cell_ijk(d, c, i, j, k);
    v[c] = (T)((double)v[c] - band_aw(bx, by, bz, comp, d, c, i, j, k, coef));
  }
}

// The projected true residual on the band, formed in FP64 and rounded once:
// r32_c = fl32((bt - At p)_c - (At Z coef)_c).  Off the band (At Z coef)_c = 0
// and r32 already holds fl32(bt - At p).  Near a component both terms are
// large and nearly cancel, so they must not be rounded separately.  p may be
// null: p = 0.
__global__ void k_defl_resid_band(const int *__restrict__ band, int nband,
                                  const int *__restrict__ comp, const double *__restrict__ bx,
                                  const double *__restrict__ by, const double *__restrict__ bz,
                                  const double *__restrict__ diag, Dims d,
                                  const double *__restrict__ coef, const double *__restrict__ p,
                                  const double *__restrict__ b, float *__restrict__ r32) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nband; e += gridDim.x * blockDim.x) {
    const size_t c = (size_t)band[e];
    int i, j, k;
    cell_ijk(d, c, i, j, k);
    const double res = p ? resid_at<double>(p, b, bx, by, bz, diag, nullptr, d, i, j, k) : b[c];
    r32[c] = (float)(res - band_aw(bx, by, bz, comp, d, c, i, j, k, coef));
  }
}

template <int W>
struct IVec16;
template <>
struct IVec16<4> {
  using V = int4;
  __device__ static int at(const V &v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
  }
};
template <>
struct IVec16<2> {
  using V = int2;
  __device__ static int at(const V &v, int i) { return i == 0 ? v.x : v.y; }
};

// z <- P^T z = z - Z coef (coef = E^-1 (A Z)^T z) on every cell of a
// component, fused with the partial sums of r . (P^T z).  16-byte accesses
// when z and r are 16-byte aligned (internal buffers always are).
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS, 4)
k_dot_zdefl(const T *__restrict__ r, T *__restrict__ z, const int *__restrict__ comp,
            const T *__restrict__ coef, size_t n, double *__restrict__ partial) {
  griddep_wait();
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int W = VT::W;
  T acc = 0;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if (aligned16(r, z)) {
    const size_t nv = n / W;
    const V *rv = reinterpret_cast<const V *>(r);
    V *zv = reinterpret_cast<V *>(z);
    const typename IVec16<W>::V *cv = reinterpret_cast<const typename IVec16<W>::V *>(comp);
    for (size_t e = tid; e < nv; e += stride) {
      const V x = rv[e];
      V y = zv[e];
      const typename IVec16<W>::V ce = cv[e];
      bool any = false;
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int m = IVec16<W>::at(ce, q);
        if (m >= 0) {
          VT::set(y, q, VT::at(y, q) - coef[m]);
          any = true;
        }
        acc = fma(VT::at(x, q), VT::at(y, q), acc);
      }
      if (any) zv[e] = y;
    }
    done = nv * W;
  }
  for (size_t e = done + tid; e < n; e += stride) {
    const int m = comp[e];
    if (m >= 0) z[e] -= coef[m];
    acc = fma(r[e], z[e], acc);
  }
  double t = block_sum((double)acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// x_c += coef[comp_c] on every cell of a component (the deflation correction)
__global__ void k_defl_add_z(double *__restrict__ x, const int *__restrict__ comp, size_t n,
                             const double *__restrict__ coef) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const int m = comp[c];
    if (m >= 0) x[c] += coef[m];
  }
}

// E -> 1/E (fixed-point sums with a fixed scale; the sums are zeroed)
__global__ void k_defl_einv(int m, unsigned long long *acc, double scale,
                            double *__restrict__ einv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double e = fx_value(acc, j, scale, true);
  einv[j] = e != 0.0 ? 1.0 / e : 0.0;
}

}  // namespace mp
