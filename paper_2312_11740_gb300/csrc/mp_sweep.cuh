// Fused red-black Gauss-Seidel sweep of the FP32 V-cycle (FP16 faces): both
// colours of one sweep in a single z-marching pass, with shared-memory halo
// staging.
//
// A sweep updates the first colour c0 from the old values of the other
// colour c1, then c1 from the new c0 values.  Done as two launches, every
// launch streams x, b and all face arrays although it updates half of the
// cells (measured: ~33 B/cell of DRAM traffic per sweep).  Here one launch
// reads x_in, b and the faces once and writes x_out once (~19 B/cell with the
// chunk overlaps), the output going to a second buffer: CTAs never read
// values that another CTA has already replaced, so the result is exactly
// that of the two in-place launches, cell for cell (same operands, same
// operation order), whatever the CTAs' relative progress.
//
// CTA tile: 64 (x) x 8 (y) cells over a chunk [z0, z1) of planes.  The CTA
// marches in z; at step k it
//   A) updates c0 on plane k over the tile and a ring of one cell around it
//      (the ring is recomputed by both neighbouring CTAs, from a two-cell
//      halo of old values), keeping the new c0 values in shared memory;
//   B) updates c1 on plane k-1 over the tile from the new c0 values of planes
//      k-2, k-1, k and writes plane k-1 (both colours) to x_out.
// One barrier per plane separates A of step k (writes plane k's c0 values)
// from B of step k+1 (reads them).  Each plane of x_in (tile + 2 ring), b,
// and the three FP16 face arrays (tile + 1 ring) is staged in a six-slot
// ring by 16-byte cp.async copies issued three planes ahead (a step reads
// the slots of planes k-1, k, k+1; the slot of k-2 is refilled with k+4);
// every copy's
// source index is wrapped on its axis, so periodic and wall axes (whose wall
// face is zero) need no special cases, and a tile that overhangs the grid
// computes wrapped copies of real cells (the stores keep only real cells).
// Each of the first 128 threads owns one 4-cell x-chunk of the tile and
// keeps its chunk's values of the previous planes (x, b, faces, new c0) in
// registers, so shared memory serves only the in-plane neighbours; a fifth
// warp updates the ring of stage A meanwhile.
//
// Requirements (checked by the host): nx a multiple of 8, x_in/x_out/b and
// the faces 16-byte aligned rows, x_in != x_out.
#pragma once

namespace mp {

constexpr int FS_TX = 64, FS_TY = 8, FS_NSLOT = 6;
constexpr int FS_OWNERS = FS_TY * (FS_TX / 4);   // threads owning a 4-cell chunk of the tile
constexpr int FS_THREADS = FS_OWNERS + 32;       // + one warp for the ring of stage A
// staged regions of one plane: rows start at y0 - 2 (x) or y0 - 1 (the
// rest), columns at x0 - 4 (x, b: 16-byte chunks of 4 floats) or x0 - 8
// (faces: 16-byte chunks of 8 halves)
constexpr int FS_XR = FS_TY + 4, FS_XC = FS_TX + 8;
constexpr int FS_BR = FS_TY + 2, FS_BC = FS_TX + 8;
constexpr int FS_HR = FS_TY + 2, FS_HYR = FS_TY + 3, FS_HC = FS_TX + 16;
constexpr int FS_X_BYTES = FS_XR * FS_XC * 4;
constexpr int FS_B_BYTES = FS_BR * FS_BC * 4;
constexpr int FS_HX_BYTES = FS_HR * FS_HC * 2;
constexpr int FS_HY_BYTES = FS_HYR * FS_HC * 2;
constexpr int FS_HZ_BYTES = FS_HR * FS_HC * 2;
constexpr int FS_SLOT_BYTES = FS_X_BYTES + FS_B_BYTES + FS_HX_BYTES + FS_HY_BYTES + FS_HZ_BYTES;
constexpr int FS_SMEM = FS_NSLOT * FS_SLOT_BYTES;
// 16-byte copy tasks of one plane, in slot order: task e fills bytes
// [16e, 16e + 16) of the slot
constexpr int FS_TX_CH = FS_XC / 4, FS_TH_CH = FS_HC / 8;  // chunks per row
constexpr int FS_E_B = FS_XR * FS_TX_CH;                   // first task of b
constexpr int FS_E_HX = FS_E_B + FS_BR * FS_TX_CH;
constexpr int FS_E_HY = FS_E_HX + FS_HR * FS_TH_CH;
constexpr int FS_E_HZ = FS_E_HY + FS_HYR * FS_TH_CH;
constexpr int FS_TASKS = FS_E_HZ + FS_HR * FS_TH_CH;
constexpr int FS_TASK_ROUNDS = (FS_TASKS + FS_THREADS - 1) / FS_THREADS;
static_assert(FS_TASKS * 16 == FS_SLOT_BYTES, "copy tasks tile the slot");
static_assert(FS_OWNERS % 32 == 0, "owner threads fill whole warps");

struct FusedArgs {
  const float *xin;  // x before the sweep (not read when zero != 0)
  float *xout;       // x after the sweep
  const float *b;    // h^2-scaled right-hand side
  const __half *hx, *hy, *hz;  // FP16 face coefficients, scaled by fs
  Dims d;
  int c0;    // colour updated first: cells with (i + j + k) & 1 == c0
  int zero;  // x_in taken as zero (first sweep of a cycle)
  float fs;
  int tiles_x, tiles_y, nchunk;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ int wrap_mod(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

// new value of one cell: the arithmetic of k_rbgs_h4, operation for operation
__device__ __forceinline__ float fs_cell(float bv, float fs, float wxl, float wxh, float wyl,
                                         float wyh, float wzl, float wzh, float xl, float xh,
                                         float yl, float yh, float zl, float zh, bool zero) {
  float s = -bv * fs;
  if (!zero) {
    s = fmaf(wxl, xl, s);
    s = fmaf(wxh, xh, s);
    s = fmaf(wyl, yl, s);
    s = fmaf(wyh, yh, s);
    s = fmaf(wzl, zl, s);
    s = fmaf(wzh, zh, s);
  }
  return __fdividef(s, ((wxl + wxh) + (wyl + wyh)) + (wzl + wzh));
}

struct FsSlot {
  float *x, *b;
  __half *hx, *hy, *hz;
  __device__ FsSlot(unsigned char *base) {
    x = reinterpret_cast<float *>(base);
    b = reinterpret_cast<float *>(base + FS_X_BYTES);
    hx = reinterpret_cast<__half *>(base + FS_X_BYTES + FS_B_BYTES);
    hy = hx + FS_HR * FS_HC;
    hz = hy + FS_HYR * FS_HC;
  }
};

__device__ __forceinline__ H4 ld_h4(const __half *p) { return *reinterpret_cast<const H4 *>(p); }
__device__ __forceinline__ float4 ld_f4(const float *p) {
  return *reinterpret_cast<const float4 *>(p);
}
__device__ __forceinline__ void f4_set(float4 &v, int q, float a) {
  if (q == 0) v.x = a; else if (q == 1) v.y = a; else if (q == 2) v.z = a; else v.w = a;
}

// Stage A for one cell of the ring, every operand from shared memory.
// (lyx, lxx): cell in the x region; the b region is one row lower, the face
// regions one row lower and four halves further right.
__device__ __forceinline__ void fs_ring_cell(const FsSlot &sm, const FsSlot &sp, const FsSlot &sk,
                                             int lyx, int lxx, float fs, bool zero) {
  const int lyh = lyx - 1, lxh = lxx + 4;
  const float wxl = __half2float(sk.hx[lyh * FS_HC + lxh]);
  const float wxh = __half2float(sk.hx[lyh * FS_HC + lxh + 1]);
  const float wyl = __half2float(sk.hy[lyh * FS_HC + lxh]);
  const float wyh = __half2float(sk.hy[(lyh + 1) * FS_HC + lxh]);
  const float wzl = __half2float(sk.hz[lyh * FS_HC + lxh]);
  const float wzh = __half2float(sp.hz[lyh * FS_HC + lxh]);
  float xl = 0.f, xh = 0.f, yl = 0.f, yh = 0.f, zl = 0.f, zh = 0.f;
  if (!zero) {
    const int c = lyx * FS_XC + lxx;
    xl = sk.x[c - 1];
    xh = sk.x[c + 1];
    yl = sk.x[c - FS_XC];
    yh = sk.x[c + FS_XC];
    zl = sm.x[c];
    zh = sp.x[c];
  }
  sk.x[lyx * FS_XC + lxx] = fs_cell(sk.b[(lyx - 1) * FS_BC + lxx], fs, wxl, wxh, wyl, wyh, wzl,
                                    wzh, xl, xh, yl, yh, zl, zh, zero);
}

// Per-plane state of an owner thread's chunk, carried between steps.
struct FsChunk {
  float4 xm1, xc;    // x_in of planes k-1, k (old values of the chunk)
  float4 c0m2, c0m1; // new c0 values of planes k-2, k-1
  float4 bm1;        // b of plane k-1
  H4 hxm1, hym1, hynm1, hzm1, hzc;  // faces of plane k-1 (x, y low, y high, z low); z low of k
  float hxem1;       // x face at i0 + 4 of plane k-1
};

// Operands of stage A for the owner's chunk on plane k that do not depend on
// the colour pattern.  Loaded (and the neighbour values exchanged between
// lanes) by every lane of the warp before the pattern-dependent code, so the
// shuffles never sit in a divergent branch.
struct FsPlaneA {
  float4 xp1, bk, yl4, yh4;  // x of plane k+1, b, x of rows j-1 and j+1
  H4 hxk, hyk, hynk, hzp;    // x faces, y faces (rows j, j+1), z faces of plane k+1
  float hxek, xl, xh;        // x face at i0 + 4; old x at i0 - 1 and i0 + 4
};

template <bool ZERO>
__device__ __forceinline__ void fs_load_a(FsPlaneA &pa, const FsChunk &st, const FsSlot &sk,
                                          const FsSlot &sp, int cx, int cb, int ch, int q) {
  pa.xp1 = ZERO ? make_float4(0.f, 0.f, 0.f, 0.f) : ld_f4(sp.x + cx);
  pa.bk = ld_f4(sk.b + cb);
  pa.hxk = ld_h4(sk.hx + ch);
  pa.hyk = ld_h4(sk.hy + ch);
  pa.hynk = ld_h4(sk.hy + ch + FS_HC);
  pa.hzp = ld_h4(sp.hz + ch);
  // x face at i0 + 4 = first face of the chunk to the right (shared memory
  // for the last chunk of a row); likewise the old x values next to the chunk
  const float hxr = __shfl_down_sync(0xffffffffu, __low2float(pa.hxk.a), 1);
  pa.hxek = q == 15 ? __half2float(sk.hx[ch + 4]) : hxr;
  pa.yl4 = pa.yh4 = make_float4(0.f, 0.f, 0.f, 0.f);
  pa.xl = pa.xh = 0.f;
  if (!ZERO) {
    pa.yl4 = ld_f4(sk.x + cx - FS_XC);
    pa.yh4 = ld_f4(sk.x + cx + FS_XC);
    const float vl = __shfl_up_sync(0xffffffffu, st.xc.w, 1);
    const float vh = __shfl_down_sync(0xffffffffu, st.xc.x, 1);
    pa.xl = q == 0 ? sk.x[cx - 1] : vl;
    pa.xh = q == 15 ? sk.x[cx + 4] : vh;
  }
}

// Stage A for the owner's chunk on plane k; O = position of the chunk's first
// c0 cell.  Returns the new c0 values (other positions 0) and stores them to
// shared memory.
template <int O, bool ZERO>
__device__ __forceinline__ float4 fs_stage_a(const FsChunk &st, const FsPlaneA &pa,
                                             const FsSlot &sk, int cx, float fs) {
  float4 c0k = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int p = O + 2 * e;
    const float wxl = h4_at(pa.hxk, p), wxh = p < 3 ? h4_at(pa.hxk, p + 1) : pa.hxek;
    const float v = fs_cell(f4_at(pa.bk, p), fs, wxl, wxh, h4_at(pa.hyk, p), h4_at(pa.hynk, p),
                            h4_at(st.hzc, p), h4_at(pa.hzp, p),
                            p > 0 ? f4_at(st.xc, p - 1) : pa.xl,
                            p < 3 ? f4_at(st.xc, p + 1) : pa.xh, f4_at(pa.yl4, p),
                            f4_at(pa.yh4, p), f4_at(st.xm1, p), f4_at(pa.xp1, p), ZERO);
    f4_set(c0k, p, v);
    sk.x[cx + p] = v;
  }
  return c0k;
}

// Stage B for the owner's chunk on plane m = k - 1; OM = position of the
// chunk's first c0 cell on plane m; (yl4, yh4, xl, xh): new c0 values of the
// in-plane neighbours.  Returns plane m's chunk.
template <int OM>
__device__ __forceinline__ float4 fs_stage_b(const FsChunk &st, const float4 &yl4,
                                             const float4 &yh4, float xl, float xh, float fs,
                                             const float4 &c0k) {
  float4 out = st.c0m1;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int p = 1 - OM + 2 * e;
    const float wxl = h4_at(st.hxm1, p), wxh = p < 3 ? h4_at(st.hxm1, p + 1) : st.hxem1;
    const float v = fs_cell(f4_at(st.bm1, p), fs, wxl, wxh, h4_at(st.hym1, p),
                            h4_at(st.hynm1, p), h4_at(st.hzm1, p), h4_at(st.hzc, p),
                            p > 0 ? f4_at(st.c0m1, p - 1) : xl, p < 3 ? f4_at(st.c0m1, p + 1) : xh,
                            f4_at(yl4, p), f4_at(yh4, p), f4_at(st.c0m2, p), f4_at(c0k, p), false);
    f4_set(out, p, v);
  }
  return out;
}

template <bool ZERO>
__global__ void __launch_bounds__(FS_THREADS, 3) k_rbgs_fused(const FusedArgs a) {
  griddep_wait();
  extern __shared__ __align__(16) unsigned char fs_smem[];
  const int tid = threadIdx.x;
  const int nx = a.d.nx, ny = a.d.ny, nz = a.d.nz;
  const int blk = blockIdx.x;
  const int tx = blk % a.tiles_x, rest = blk / a.tiles_x;
  const int x0 = tx * FS_TX, y0 = (rest % a.tiles_y) * FS_TY, cz = rest / a.tiles_y;
  const int z0 = (int)((long long)cz * nz / a.nchunk);
  const int z1 = (int)((long long)(cz + 1) * nz / a.nchunk);
  const size_t plane = (size_t)nx * ny;

  // this thread's copy tasks: source address inside plane 0, the class of
  // planes it is copied for (0: x, 1: b and x/y faces, 2: z faces; -1 none)
  // and its element size
  const char *tsrc[FS_TASK_ROUNDS];
  int tcls[FS_TASK_ROUNDS];
  bool tf32[FS_TASK_ROUNDS];
#pragma unroll
  for (int u = 0; u < FS_TASK_ROUNDS; ++u) {
    const int e = tid + u * FS_THREADS;
    int cls = -1, row = 0, col = 0;
    const char *base = nullptr;
    bool f32 = true;
    if (e < FS_E_B) {
      cls = ZERO ? -1 : 0;
      base = reinterpret_cast<const char *>(a.xin);
      row = y0 - 2 + e / FS_TX_CH;
      col = x0 - 4 + 4 * (e % FS_TX_CH);
    } else if (e < FS_E_HX) {
      cls = 1;
      base = reinterpret_cast<const char *>(a.b);
      row = y0 - 1 + (e - FS_E_B) / FS_TX_CH;
      col = x0 - 4 + 4 * ((e - FS_E_B) % FS_TX_CH);
    } else if (e < FS_TASKS) {
      const int first = e < FS_E_HY ? FS_E_HX : (e < FS_E_HZ ? FS_E_HY : FS_E_HZ);
      cls = e < FS_E_HZ ? 1 : 2;
      base = reinterpret_cast<const char *>(e < FS_E_HY ? a.hx : (e < FS_E_HZ ? a.hy : a.hz));
      f32 = false;
      row = y0 - 1 + (e - first) / FS_TH_CH;
      col = x0 - 8 + 8 * ((e - first) % FS_TH_CH);
    }
    tcls[u] = cls;
    tf32[u] = f32;
    tsrc[u] = cls < 0 ? nullptr
                      : base + ((size_t)wrap_mod(row, ny) * nx + wrap_mod(col, nx)) * (f32 ? 4 : 2);
  }
  // issue the copies of plane p (wrapped: pk) into slot s: x on
  // [z0-2, z1+1], b and the x/y faces on [z0-1, z1], z faces on
  // [z0-1, z1+1]; always one commit group
  auto issue = [&](int p, int pk, int s) {
    if (p <= z1 + 1) {
      const size_t o4 = (size_t)pk * plane * 4, o2 = o4 >> 1;
      const unsigned en = 1u | ((p >= z0 - 1 && p <= z1) ? 2u : 0u) | (p >= z0 - 1 ? 4u : 0u);
      unsigned char *slot = fs_smem + s * FS_SLOT_BYTES + 16 * tid;
#pragma unroll
      for (int u = 0; u < FS_TASK_ROUNDS; ++u)
        if (tcls[u] >= 0 && ((en >> tcls[u]) & 1u))
          cp_async16(slot + 16 * FS_THREADS * u, tsrc[u] + (tf32[u] ? o4 : o2));
    }
    cp_async_commit();
  };
  // slot of plane p is (p - z0 + 2) mod FS_NSLOT
  for (int p = z0 - 2; p <= z0 + 2; ++p) issue(p, wrap_mod(p, nz), p - z0 + 2);

  // owner threads: warp w takes rows w%2 + 4(w/2) and that + 2 (both of one
  // parity, so the colour pattern of a chunk is the same across the warp);
  // 16 chunks per row
  const int w = tid >> 5, lane = tid & 31;
  const int r = (w & 1) + 4 * (w >> 1) + 2 * (lane >> 4), q = lane & 15;
  const int j = y0 + r, i0 = x0 + 4 * q;
  const int jj = j % ny;
  const bool owner = tid < FS_OWNERS && i0 < nx && j < ny;
  const int cx = (r + 2) * FS_XC + 4 * q + 4;  // chunk in the x region
  const int cb = (r + 1) * FS_BC + 4 * q + 4, ch = (r + 1) * FS_HC + 4 * q + 8;
  FsChunk st;
  st.xm1 = st.xc = st.c0m2 = st.c0m1 = st.bm1 = make_float4(0.f, 0.f, 0.f, 0.f);
  st.hxm1 = st.hym1 = st.hynm1 = st.hzm1 = st.hzc = H4{};
  st.hxem1 = 0.f;

  int kk = wrap_mod(z0 - 1, nz), k4 = wrap_mod(z0 + 3, nz);  // planes k and k+4, wrapped
  int s = 1;                                                  // slot of plane k
  for (int k = z0 - 1; k <= z1; ++k) {
    cp_async_wait<2>();  // planes up to k+1 have landed (this thread's copies)
    __syncthreads();     // ... everyone's; step k-1 is done with the slot refilled below
    const int sm_i = s == 0 ? FS_NSLOT - 1 : s - 1, sp_i = s == FS_NSLOT - 1 ? 0 : s + 1;
    issue(k + 4, k4, s >= 2 ? s - 2 : s + FS_NSLOT - 2);
    k4 = k4 + 1 == nz ? 0 : k4 + 1;
    const FsSlot sk(fs_smem + s * FS_SLOT_BYTES), sm(fs_smem + sm_i * FS_SLOT_BYTES),
        sp(fs_smem + sp_i * FS_SLOT_BYTES);
    if (tid >= FS_OWNERS) {
      // ---- stage A on the ring: rows y0-1 and y0+8 (one chunk per lane), then
      // columns x0-1 and x0+64 (one cell per lane); cells of colour c0 only
      {
        const int ry = lane < 16 ? 1 : FS_TY + 2, qq = lane & 15;  // x-region row of y0-1 / y0+8
        const int ring_j = wrap_mod(y0 - 2 + ry, ny);
        const int o = (ring_j + kk + a.c0) & 1;
#pragma unroll
        for (int e = 0; e < 2; ++e)
          fs_ring_cell(sm, sp, sk, ry, 4 * qq + 4 + o + 2 * e, a.fs, ZERO);
      }
      if (lane < 20) {
        const int ry = 1 + lane % 10, rx = lane < 10 ? 3 : FS_TX + 4;  // x-region row/column
        const int ring_i = wrap_mod(x0 - 4 + rx, nx), ring_j = wrap_mod(y0 - 2 + ry, ny);
        if (((ring_i + ring_j + kk) & 1) == a.c0) fs_ring_cell(sm, sp, sk, ry, rx, a.fs, ZERO);
      }
    } else {
      if (k == z0 - 1) {  // first plane: prime the chunk state from shared memory
        if (!ZERO) {
          st.xm1 = ld_f4(sm.x + cx);
          st.xc = ld_f4(sk.x + cx);
        }
        st.hzc = ld_h4(sk.hz + ch);
      }
      // ---- stage A: c0 on plane k, this thread's chunk (wrapped copies of
      // real cells included: the stores below keep only real cells).  The
      // colour pattern is uniform across the warp except in a tile that
      // overhangs an odd wall axis; the branch then diverges, harmlessly
      FsPlaneA pa;
      fs_load_a<ZERO>(pa, st, sk, sp, cx, cb, ch, q);
      const float4 c0k = ((jj + kk + a.c0) & 1) ? fs_stage_a<1, ZERO>(st, pa, sk, cx, a.fs)
                                                : fs_stage_a<0, ZERO>(st, pa, sk, cx, a.fs);
      // ---- stage B: c1 on plane m = k - 1 from the new c0 values; store plane m
      if (k - 1 >= z0) {
        const int mm = kk == 0 ? nz - 1 : kk - 1;
        const float4 yl4 = ld_f4(sm.x + cx - FS_XC), yh4 = ld_f4(sm.x + cx + FS_XC);
        const float vl = __shfl_up_sync(0xffffffffu, st.c0m1.w, 1);
        const float vh = __shfl_down_sync(0xffffffffu, st.c0m1.x, 1);
        const float xl = q == 0 ? sm.x[cx - 1] : vl, xh = q == 15 ? sm.x[cx + 4] : vh;
        const float4 out = ((jj + mm + a.c0) & 1) ? fs_stage_b<1>(st, yl4, yh4, xl, xh, a.fs, c0k)
                                                  : fs_stage_b<0>(st, yl4, yh4, xl, xh, a.fs, c0k);
        if (owner)
          *reinterpret_cast<float4 *>(a.xout + (size_t)mm * plane + (size_t)j * nx + i0) = out;
      }
      // ---- the chunk state moves to the next plane
      st.xm1 = st.xc;
      st.xc = pa.xp1;
      st.c0m2 = st.c0m1;
      st.c0m1 = c0k;
      st.bm1 = pa.bk;
      st.hxm1 = pa.hxk;
      st.hxem1 = pa.hxek;
      st.hym1 = pa.hyk;
      st.hynm1 = pa.hynk;
      st.hzm1 = st.hzc;
      st.hzc = pa.hzp;
    }
    kk = kk + 1 == nz ? 0 : kk + 1;
    s = sp_i;
  }
  cp_async_wait<0>();
}

}  // namespace mp
