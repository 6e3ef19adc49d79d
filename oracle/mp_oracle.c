/*
 * FP64 CPU oracle for the variable-density pressure-Poisson solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * The paper (Section 2) fixes a staggered-grid, finite-difference,
 * fractional-step projection method: vectors on faces, scalars at cell
 * centres, a level set phi that is positive in gas and negative in liquid
 * (Fig. 2 caption), variable density from phi (varDens configuration,
 * Section 3) and a multigrid Poisson solve (Grid_solvePoisson, Section 3).
 * It prints no formulas for the solve; the discretisation written out here
 * is the published ghost-fluid method for a variable-coefficient Poisson
 * equation with a pressure jump [p] = sigma*kappa across the interface
 * (Liu, Fedkiw & Kang 2000; Kang, Fedkiw & Liu 2000):
 *
 *   A p = b,  (A p)_c = sum_faces beta_f (p_nb - p_c) / h^2,
 *   b = rhs + J - mean(rhs + J),   gauge mean(p) = 0.
 *
 * Boundaries: one code per axis (bc[a]): 0 periodic; 1 wall or inflow on
 * both sides (zero normal pressure gradient: the face carries no pressure
 * flux); 2 outflow on both sides (p = 0 on the boundary face); 3 wall/inflow
 * on the low side and outflow on the high side; 4 the reverse.  The paper
 * sets boundary types per side (xl_boundary_type / xr_boundary_type with
 * inflow_ins / outflow_ins in its runtime-parameter TOML figure, Section 4);
 * an outflow face holds p = 0 through an antisymmetric ghost, p_ghost =
 * -p_cell, the cell-centred form of that condition.  With an outflow side
 * the operator has no null space: no mean projection and no gauge.
 *
 * Storage here is deliberately different from the CUDA path: every axis
 * keeps n+1 faces (face f between cells f-1 and f); on a periodic axis
 * faces 0 and n are the same physical face, on a wall axis both are walls
 * with beta = 0, on an outflow side the boundary face holds the coefficient
 * 1/rho of the cell next to it (its ghost lies in the same fluid).  Cell
 * arrays are (nz, ny, nx), x fastest.
 *
 * Entry points are plain loops, one formula at a time; nothing is blocked,
 * fused or reordered beyond the definitions.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)ny * (size_t)(k)))
/* face arrays: fx (nz, ny, nx+1), fy (nz, ny+1, nx), fz (nz+1, ny, nx) */
#define FX(i, j, k) ((size_t)(i) + (size_t)(nx + 1) * ((size_t)(j) + (size_t)ny * (size_t)(k)))
#define FY(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)(ny + 1) * (size_t)(k)))
#define FZ(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)ny * (size_t)(k)))

#define PER(bc, a) ((bc)[a] == 0)
#define DLO(bc, a) ((bc)[a] == 2 || (bc)[a] == 4) /* outflow on the low side */
#define DHI(bc, a) ((bc)[a] == 2 || (bc)[a] == 3) /* outflow on the high side */

static int any_outflow(const int bc[3]) {
  return DLO(bc, 0) || DHI(bc, 0) || DLO(bc, 1) || DHI(bc, 1) || DLO(bc, 2) || DHI(bc, 2);
}

/* Neighbour index along one axis: periodic wrap, or mirror at a wall
 * (even reflection: ghost -1 -> 0, ghost n -> n-1). */
static int ghost(int i, int n, int periodic) {
  if (i < 0) return periodic ? i + n : -1 - i;
  if (i >= n) return periodic ? i - n : 2 * n - 1 - i;
  return i;
}

static int is_gas(double phi) { return phi > 0.0; } /* phi = 0 counts as liquid */

/*
 * Curvature kappa = -div(grad phi / |grad phi|) at cell centres, from
 * second-order central differences of phi (mirror ghosts at walls):
 *   kappa = -[phi_x^2 (phi_yy + phi_zz) + phi_y^2 (phi_xx + phi_zz)
 *             + phi_z^2 (phi_xx + phi_yy)
 *             - 2 (phi_x phi_y phi_xy + phi_x phi_z phi_xz + phi_y phi_z phi_yz)]
 *           / |grad phi|^3,
 * |grad phi| floored at 1e-12, result clamped to |kappa| <= 1/h.
 * With phi > 0 in gas a spherical bubble of radius R has kappa = +2/R.
 * Surface tension enters through the jump [p] = sigma kappa (the paper's
 * mph_invWeber parameter of the runtime-parameter TOML figure, Section 4;
 * MultiphaseMain, Section 3).
 */
void oracle_curvature(int nx, int ny, int nz, double h, const int bc[3],
                      const double *phi, double *kappa) {
  const int periodic[3] = {PER(bc, 0), PER(bc, 1), PER(bc, 2)};
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int im = ghost(i - 1, nx, periodic[0]), ip = ghost(i + 1, nx, periodic[0]);
        int jm = ghost(j - 1, ny, periodic[1]), jp = ghost(j + 1, ny, periodic[1]);
        int km = ghost(k - 1, nz, periodic[2]), kp = ghost(k + 1, nz, periodic[2]);
        double c = phi[IDX(i, j, k)];
        double px = (phi[IDX(ip, j, k)] - phi[IDX(im, j, k)]) / (2.0 * h);
        double py = (phi[IDX(i, jp, k)] - phi[IDX(i, jm, k)]) / (2.0 * h);
        double pz = (phi[IDX(i, j, kp)] - phi[IDX(i, j, km)]) / (2.0 * h);
        double pxx = (phi[IDX(ip, j, k)] - 2.0 * c + phi[IDX(im, j, k)]) / (h * h);
        double pyy = (phi[IDX(i, jp, k)] - 2.0 * c + phi[IDX(i, jm, k)]) / (h * h);
        double pzz = (phi[IDX(i, j, kp)] - 2.0 * c + phi[IDX(i, j, km)]) / (h * h);
        double pxy = (phi[IDX(ip, jp, k)] - phi[IDX(ip, jm, k)] - phi[IDX(im, jp, k)] +
                      phi[IDX(im, jm, k)]) / (4.0 * h * h);
        double pxz = (phi[IDX(ip, j, kp)] - phi[IDX(ip, j, km)] - phi[IDX(im, j, kp)] +
                      phi[IDX(im, j, km)]) / (4.0 * h * h);
        double pyz = (phi[IDX(i, jp, kp)] - phi[IDX(i, jp, km)] - phi[IDX(i, jm, kp)] +
                      phi[IDX(i, jm, km)]) / (4.0 * h * h);
        double g = sqrt(px * px + py * py + pz * pz);
        if (g < 1e-12) g = 1e-12;
        double num = px * px * (pyy + pzz) + py * py * (pxx + pzz) + pz * pz * (pxx + pyy) -
                     2.0 * (px * py * pxy + px * pz * pxz + py * pz * pyz);
        double kap = -num / (g * g * g);
        if (kap > 1.0 / h) kap = 1.0 / h;
        if (kap < -1.0 / h) kap = -1.0 / h;
        kappa[IDX(i, j, k)] = kap;
      }
}

/*
 * Ghost-fluid face coefficient between a cell a (low side) and b (high side)
 * (Liu, Fedkiw & Kang 2000; variable density from phi, varDens):
 * both cells on one side -> beta = 1/rho(side); otherwise the interface sits
 * at fraction theta = |phi_a| / (|phi_a| + |phi_b|) of the way from a to b,
 * the two fluid layers act in series and
 *   beta = 1 / (theta rho(a) + (1 - theta) rho(b)).
 */
static double face_beta(double pa, double pb, double rho_l, double rho_g) {
  double ra = is_gas(pa) ? rho_g : rho_l;
  double rb = is_gas(pb) ? rho_g : rho_l;
  if (is_gas(pa) == is_gas(pb)) return 1.0 / ra;
  double theta = fabs(pa) / (fabs(pa) + fabs(pb));
  return 1.0 / (theta * ra + (1.0 - theta) * rb);
}

/* Coefficient of an outflow boundary face next to cell value pc: the ghost
 * cell beyond the face lies in the same fluid as the cell. */
static double out_beta(double pc, double rho_l, double rho_g) {
  return 1.0 / (is_gas(pc) ? rho_g : rho_l);
}

/* Face coefficients for every face; walls get beta = 0 (no flux), outflow
 * faces the coefficient of the fluid of their cell. */
void oracle_faces(int nx, int ny, int nz, const int bc[3], const double *phi,
                  double rho_l, double rho_g, double *fx, double *fy, double *fz) {
  const int periodic[3] = {PER(bc, 0), PER(bc, 1), PER(bc, 2)};
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        double v;
        if (i == 0 || i == nx) {
          v = periodic[0] ? face_beta(phi[IDX(nx - 1, j, k)], phi[IDX(0, j, k)], rho_l, rho_g) : 0.0;
          if (i == 0 && DLO(bc, 0)) v = out_beta(phi[IDX(0, j, k)], rho_l, rho_g);
          if (i == nx && DHI(bc, 0)) v = out_beta(phi[IDX(nx - 1, j, k)], rho_l, rho_g);
        } else {
          v = face_beta(phi[IDX(i - 1, j, k)], phi[IDX(i, j, k)], rho_l, rho_g);
        }
        fx[FX(i, j, k)] = v;
      }
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double v;
        if (j == 0 || j == ny) {
          v = periodic[1] ? face_beta(phi[IDX(i, ny - 1, k)], phi[IDX(i, 0, k)], rho_l, rho_g) : 0.0;
          if (j == 0 && DLO(bc, 1)) v = out_beta(phi[IDX(i, 0, k)], rho_l, rho_g);
          if (j == ny && DHI(bc, 1)) v = out_beta(phi[IDX(i, ny - 1, k)], rho_l, rho_g);
        } else {
          v = face_beta(phi[IDX(i, j - 1, k)], phi[IDX(i, j, k)], rho_l, rho_g);
        }
        fy[FY(i, j, k)] = v;
      }
#pragma omp parallel for schedule(static)
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double v;
        if (k == 0 || k == nz) {
          v = periodic[2] ? face_beta(phi[IDX(i, j, nz - 1)], phi[IDX(i, j, 0)], rho_l, rho_g) : 0.0;
          if (k == 0 && DLO(bc, 2)) v = out_beta(phi[IDX(i, j, 0)], rho_l, rho_g);
          if (k == nz && DHI(bc, 2)) v = out_beta(phi[IDX(i, j, nz - 1)], rho_l, rho_g);
        } else {
          v = face_beta(phi[IDX(i, j, k - 1)], phi[IDX(i, j, k)], rho_l, rho_g);
        }
        fz[FZ(i, j, k)] = v;
      }
}

/*
 * Pressure jump across the face from a to b: [p]_{a->b} = p(b side) - p(a side)
 * at the interface.  With [p] = p_gas - p_liquid = sigma kappa_G it is
 * +sigma kappa_G when b is gas, -sigma kappa_G when b is liquid, and 0 on
 * faces that do not cross the interface.  kappa_G interpolates the cell
 * curvatures linearly to the interface point:
 *   kappa_G = (|phi_b| kappa_a + |phi_a| kappa_b) / (|phi_a| + |phi_b|).
 */
static double face_jump(double pa, double pb, double ka, double kb, double sigma) {
  if (is_gas(pa) == is_gas(pb)) return 0.0;
  double kg = (fabs(pb) * ka + fabs(pa) * kb) / (fabs(pa) + fabs(pb));
  return is_gas(pb) ? sigma * kg : -sigma * kg;
}

/*
 * Jump source J of the ghost-fluid discretisation (Kang, Fedkiw & Liu 2000):
 * the flux across a face a->b is beta (p_b - p_a - [p]_{a->b}) / h, so every
 * interface face adds +beta [p]_{a->b} / h^2 to row a and -beta [p]_{a->b} / h^2
 * to row b.  J sums to zero.  Face loops visit each physical face once.
 */
void oracle_jump(int nx, int ny, int nz, double h, const int bc[3], const double *phi,
                 const double *kappa, const double *fx, const double *fy, const double *fz,
                 double sigma, double *J) {
  const int periodic[3] = {PER(bc, 0), PER(bc, 1), PER(bc, 2)};
  size_t n = (size_t)nx * ny * nz;
  memset(J, 0, n * sizeof(double));
  double ih2 = 1.0 / (h * h);
  /* serial: each face updates two rows */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t b = IDX(i, j, k);
        /* low x face of cell b: between a = (i-1) and b */
        if (i > 0 || periodic[0]) {
          size_t a = IDX(i > 0 ? i - 1 : nx - 1, j, k);
          double jp = face_jump(phi[a], phi[b], kappa[a], kappa[b], sigma);
          double t = fx[FX(i, j, k)] * jp * ih2;
          J[a] += t;
          J[b] -= t;
        }
        if (j > 0 || periodic[1]) {
          size_t a = IDX(i, j > 0 ? j - 1 : ny - 1, k);
          double jp = face_jump(phi[a], phi[b], kappa[a], kappa[b], sigma);
          double t = fy[FY(i, j, k)] * jp * ih2;
          J[a] += t;
          J[b] -= t;
        }
        if (k > 0 || periodic[2]) {
          size_t a = IDX(i, j, k > 0 ? k - 1 : nz - 1);
          double jp = face_jump(phi[a], phi[b], kappa[a], kappa[b], sigma);
          double t = fz[FZ(i, j, k)] * jp * ih2;
          J[a] += t;
          J[b] -= t;
        }
      }
}

/*
 * Phase change (evaporation; the MultiphaseEvap unit of Section 3, which
 * adds mass transfer at the interface to the main multiphase unit).  The
 * paper prints no formulas; this is the ghost-fluid reading.  A mass flux
 * mdot (per unit interface area, liquid -> gas) makes the normal velocity
 * jump, [u.n] = u_gas.n - u_liquid.n = mdot [1/rho], [1/rho] = 1/rho_g -
 * 1/rho_l, n the normal from liquid into gas.  With u = u* - beta grad p
 * (Delta t = 1) and u* continuous, the pressure flux jumps by
 *   B = [beta dp/dn] = beta_g dp_g/dn - beta_l dp_l/dn = -mdot [1/rho],
 * a quantity that does not depend on which side of a face is which.
 *
 * On a face between cells a and b with the interface at fraction theta_a =
 * |phi_a| / (|phi_a| + |phi_b|) of the way from a (theta_b = 1 - theta_a),
 * p linear on each side with the two jump conditions gives the flux on a's
 * side F_a = beta (p_b - p_a - [p]_{a->b}) / h - beta theta_b rho_b B and on
 * b's side F_b = F_a + B = beta (p_b - p_a - [p]_{a->b}) / h + beta theta_a
 * rho_a B (beta the face coefficient, 1 / (theta_a rho_a + theta_b rho_b)).
 * Each row takes the flux of its own side, so the face adds
 *   beta theta_b rho_b B / h  to row a,   beta theta_a rho_a B / h  to row b,
 * B / h in total: the volume the phase change creates.  The interface value
 * of mdot interpolates the cell values like the curvature:
 *   mdot_G = (|phi_b| mdot_a + |phi_a| mdot_b) / (|phi_a| + |phi_b|).
 */
static double face_flux_jump(double pa, double pb, double ma, double mb, double jinv) {
  if (is_gas(pa) == is_gas(pb)) return 0.0;
  double mg = (fabs(pb) * ma + fabs(pa) * mb) / (fabs(pa) + fabs(pb));
  return -mg * jinv;
}

/* beta theta_nb rho_nb: the part of B that the row of cell c carries for its
 * face to nb (the fraction of the c-nb segment in nb's fluid, times nb's
 * density, times the face coefficient). */
static double flux_share(double pc, double pnb, double beta, double rho_l, double rho_g) {
  double rnb = is_gas(pnb) ? rho_g : rho_l;
  return beta * fabs(pnb) / (fabs(pc) + fabs(pnb)) * rnb;
}

/* J += the phase-change flux-jump source of every interface face (above);
 * mdot: cell values (N). */
void oracle_flux_jump(int nx, int ny, int nz, double h, const int bc[3], const double *phi,
                      const double *mdot, const double *fx, const double *fy, const double *fz,
                      double rho_l, double rho_g, double *J) {
  const int periodic[3] = {PER(bc, 0), PER(bc, 1), PER(bc, 2)};
  const double jinv = 1.0 / rho_g - 1.0 / rho_l;
  /* serial: each face updates two rows */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t b = IDX(i, j, k);
        size_t a[3] = {0, 0, 0};
        int has[3] = {i > 0 || periodic[0], j > 0 || periodic[1], k > 0 || periodic[2]};
        double beta[3] = {fx[FX(i, j, k)], fy[FY(i, j, k)], fz[FZ(i, j, k)]};
        a[0] = IDX(i > 0 ? i - 1 : nx - 1, j, k);
        a[1] = IDX(i, j > 0 ? j - 1 : ny - 1, k);
        a[2] = IDX(i, j, k > 0 ? k - 1 : nz - 1);
        for (int ax = 0; ax < 3; ++ax) {
          if (!has[ax]) continue;
          double B = face_flux_jump(phi[a[ax]], phi[b], mdot[a[ax]], mdot[b], jinv);
          if (B == 0.0) continue;
          J[a[ax]] += flux_share(phi[a[ax]], phi[b], beta[ax], rho_l, rho_g) * B / h;
          J[b] += flux_share(phi[b], phi[a[ax]], beta[ax], rho_l, rho_g) * B / h;
        }
      }
}

/*
 * The phase-change part of the velocity correction.  A face crossing the
 * interface has a liquid-side and a gas-side velocity (they differ by the
 * jump mdot [1/rho]); the face stores the liquid-side one, u*_f - F_liquid
 * (F_a when a is liquid, F_b when b is): on top of oracle_project's
 * correction that adds +beta theta_b rho_b B when a is liquid and
 * -beta theta_a rho_a B when b is.  The gas-side velocity is the stored one
 * plus the jump.  Updates ux, uy, uz (n+1 faces per axis) in place.
 */
void oracle_project_flux(int nx, int ny, int nz, const int bc[3], const double *phi,
                         const double *mdot, const double *fx, const double *fy,
                         const double *fz, double rho_l, double rho_g, double *ux, double *uy,
                         double *uz) {
  const int periodic[3] = {PER(bc, 0), PER(bc, 1), PER(bc, 2)};
  const double jinv = 1.0 / rho_g - 1.0 / rho_l;
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i)
        for (int ax = 0; ax < 3; ++ax) {
          int idx3[3] = {i, j, k}, n3[3] = {nx, ny, nz};
          int in = 1; /* the face exists on this axis (other indices in range) */
          for (int q = 0; q < 3; ++q)
            if (q != ax && idx3[q] >= n3[q]) in = 0;
          if (!in) continue;
          int f = idx3[ax];
          if ((f == 0 || f == n3[ax]) && !periodic[ax]) continue; /* boundary face */
          int lo[3] = {i, j, k}, hi[3] = {i, j, k};
          lo[ax] = f == 0 ? n3[ax] - 1 : f - 1;
          hi[ax] = f == n3[ax] ? 0 : f;
          size_t a = IDX(lo[0], lo[1], lo[2]), b = IDX(hi[0], hi[1], hi[2]);
          double B = face_flux_jump(phi[a], phi[b], mdot[a], mdot[b], jinv);
          if (B == 0.0) continue;
          double *u = ax == 0 ? &ux[FX(i, j, k)] : (ax == 1 ? &uy[FY(i, j, k)] : &uz[FZ(i, j, k)]);
          double beta = ax == 0 ? fx[FX(i, j, k)] : (ax == 1 ? fy[FY(i, j, k)] : fz[FZ(i, j, k)]);
          if (!is_gas(phi[a]))
            *u += flux_share(phi[a], phi[b], beta, rho_l, rho_g) * B;
          else
            *u -= flux_share(phi[b], phi[a], beta, rho_l, rho_g) * B;
        }
}

/* The cell across the low (low = 1) or high face of cell i on an axis of n
 * cells with boundary code `code`, given inb = i - 1 or i + 1: its index
 * inside the grid (wrapped on a periodic axis), -1 at an outflow face (the
 * ghost value is -x_c), -2 at a wall (the face coefficient is zero; the
 * cell's own value is used). */
static int across(int inb, int n, int code, int low) {
  if (inb >= 0 && inb < n) return inb;
  if (code == 0) return inb < 0 ? n - 1 : 0;
  if (low ? (code == 2 || code == 4) : (code == 2 || code == 3)) return -1;
  return -2;
}
static double value(int m, double xin, double xc) { return m >= 0 ? xin : (m == -1 ? -xc : xc); }

/* y = A x, (A x)_c = sum over the six faces of beta_f (x_nb - x_c) / h^2,
 * x_nb the neighbour's value or the ghost value at a boundary face. */
void oracle_apply(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
                  const double *fy, const double *fz, const double *x, double *y) {
  double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xc = x[IDX(i, j, k)];
        int a;
        double s = 0.0;
        a = across(i - 1, nx, bc[0], 1);
        s += fx[FX(i, j, k)] * (value(a, a >= 0 ? x[IDX(a, j, k)] : 0.0, xc) - xc);
        a = across(i + 1, nx, bc[0], 0);
        s += fx[FX(i + 1, j, k)] * (value(a, a >= 0 ? x[IDX(a, j, k)] : 0.0, xc) - xc);
        a = across(j - 1, ny, bc[1], 1);
        s += fy[FY(i, j, k)] * (value(a, a >= 0 ? x[IDX(i, a, k)] : 0.0, xc) - xc);
        a = across(j + 1, ny, bc[1], 0);
        s += fy[FY(i, j + 1, k)] * (value(a, a >= 0 ? x[IDX(i, a, k)] : 0.0, xc) - xc);
        a = across(k - 1, nz, bc[2], 1);
        s += fz[FZ(i, j, k)] * (value(a, a >= 0 ? x[IDX(i, j, a)] : 0.0, xc) - xc);
        a = across(k + 1, nz, bc[2], 0);
        s += fz[FZ(i, j, k + 1)] * (value(a, a >= 0 ? x[IDX(i, j, a)] : 0.0, xc) - xc);
        y[IDX(i, j, k)] = s * ih2;
      }
}

/* Diagonal of -A: the six face coefficients over h^2, an outflow face twice
 * (its ghost value -x_c adds -2 beta x_c to (A x)_c). */
static void neg_diag(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
                     const double *fy, const double *fz, double *d) {
  double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double w[6] = {fx[FX(i, j, k)], fx[FX(i + 1, j, k)], fy[FY(i, j, k)],
                       fy[FY(i, j + 1, k)], fz[FZ(i, j, k)], fz[FZ(i, j, k + 1)]};
        int m[6] = {across(i - 1, nx, bc[0], 1), across(i + 1, nx, bc[0], 0),
                    across(j - 1, ny, bc[1], 1), across(j + 1, ny, bc[1], 0),
                    across(k - 1, nz, bc[2], 1), across(k + 1, nz, bc[2], 0)};
        double s = 0.0;
        for (int f = 0; f < 6; ++f) s += m[f] == -1 ? 2.0 * w[f] : w[f];
        d[IDX(i, j, k)] = s * ih2;
      }
}

static double dot(size_t n, const double *a, const double *b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* r = b - A x; returns ||r||_2. */
double oracle_residual(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
                       const double *fy, const double *fz, const double *b, const double *x,
                       double *r) {
  size_t n = (size_t)nx * ny * nz;
  oracle_apply(nx, ny, nz, h, bc, fx, fy, fz, x, r);
#pragma omp parallel for schedule(static)
  for (size_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  return sqrt(dot(n, r, r));
}

/* Remove the mean (the operator annihilates constants: periodic/wall
 * boundaries leave p determined up to a constant; gauge mean(p) = 0). */
void oracle_remove_mean(size_t n, double *x) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += x[i];
  s /= (double)n;
  for (size_t i = 0; i < n; ++i) x[i] -= s;
}

/* y = M x with M = -A (symmetric positive semidefinite). */
static void apply_neg(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
                      const double *fy, const double *fz, const double *x, double *y) {
  size_t n = (size_t)nx * ny * nz;
  oracle_apply(nx, ny, nz, h, bc, fx, fy, fz, x, y);
#pragma omp parallel for schedule(static)
  for (size_t i = 0; i < n; ++i) y[i] = -y[i];
}

/* rho = f - M x, returns ||rho||_2 */
static double neg_residual(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
                           const double *fy, const double *fz, const double *f, const double *x,
                           double *rho) {
  size_t n = (size_t)nx * ny * nz;
  apply_neg(nx, ny, nz, h, bc, fx, fy, fz, x, rho);
#pragma omp parallel for schedule(static)
  for (size_t i = 0; i < n; ++i) rho[i] = f[i] - rho[i];
  return sqrt(dot(n, rho, rho));
}

/*
 * Jacobi-preconditioned conjugate gradients (textbook PCG) on M x = f with
 * M = -A, f = -b: M is symmetric positive semidefinite with null space the
 * constants (periodic and wall boundaries; b must then be mean-free so the
 * system is consistent), or positive definite with an outflow side.
 * x is the initial guess on entry and the solution on exit (mean-free when
 * the system is singular).  Stops when ||b - A x|| <= tol ||b||; the
 * recurrence residual is replaced by the true one every 50 iterations and
 * checked again at the end.  Returns iterations, or -1 if maxit was hit;
 * *relres gets the final relative residual.
 */
int oracle_cg(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
              const double *fy, const double *fz, const double *b, double *x, double tol,
              int maxit, double *relres) {
  size_t n = (size_t)nx * ny * nz;
  double *f = malloc(n * sizeof(double)), *rho = malloc(n * sizeof(double));
  double *z = malloc(n * sizeof(double)), *p = malloc(n * sizeof(double));
  double *q = malloc(n * sizeof(double)), *d = malloc(n * sizeof(double));
  neg_diag(nx, ny, nz, h, bc, fx, fy, fz, d);
  for (size_t i = 0; i < n; ++i) f[i] = -b[i];
  double fn = sqrt(dot(n, f, f));
  int status = -1;
  if (fn == 0.0) {
    memset(x, 0, n * sizeof(double));
    status = 0;
  } else {
    double rn = neg_residual(nx, ny, nz, h, bc, fx, fy, fz, f, x, rho);
    double rz_old = 0.0;
    for (int it = 0; it <= maxit; ++it) {
      if (rn <= tol * fn) { status = it; break; }
      if (it == maxit) break;
#pragma omp parallel for schedule(static)
      for (size_t i = 0; i < n; ++i) z[i] = rho[i] / d[i];
      double rz = dot(n, rho, z);
      if (it == 0) {
        memcpy(p, z, n * sizeof(double));
      } else {
        double beta = rz / rz_old;
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      }
      rz_old = rz;
      apply_neg(nx, ny, nz, h, bc, fx, fy, fz, p, q);
      double alpha = rz / dot(n, p, q);
#pragma omp parallel for schedule(static)
      for (size_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        rho[i] -= alpha * q[i];
      }
      if ((it + 1) % 50 == 0)
        rn = neg_residual(nx, ny, nz, h, bc, fx, fy, fz, f, x, rho);
      else
        rn = sqrt(dot(n, rho, rho));
    }
  }
  if (!any_outflow(bc)) oracle_remove_mean(n, x);
  double tn = neg_residual(nx, ny, nz, h, bc, fx, fy, fz, f, x, rho);
  *relres = fn > 0.0 ? tn / fn : 0.0;
  if (status >= 0 && tn > tol * fn) status = -1;
  free(f); free(rho); free(z); free(p); free(q); free(d);
  return status;
}

/*
 * Lexicographic Gauss-Seidel for small grids: each cell in turn takes
 *   x_c = (sum_f beta_f x_nb - h^2 b_c) / sum_f beta_f,
 * i.e. row c of A x = b solved for x_c; an outflow face's ghost value -x_c
 * moves to the left-hand side (twice its coefficient in the denominator,
 * nothing in the numerator).  Sweeps until ||b - A x|| <= tol ||b||.
 */
int oracle_gs(int nx, int ny, int nz, double h, const int bc[3], const double *fx,
              const double *fy, const double *fz, const double *b, double *x, double tol,
              int maxsweeps, double *relres) {
  size_t n = (size_t)nx * ny * nz;
  double *r = malloc(n * sizeof(double));
  double bn = sqrt(dot(n, b, b));
  int status = -1;
  for (int s = 0; s <= maxsweeps; ++s) {
    double rn = oracle_residual(nx, ny, nz, h, bc, fx, fy, fz, b, x, r);
    if (rn <= tol * bn) { status = s; break; }
    if (s == maxsweeps) break;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double w[6] = {fx[FX(i, j, k)], fx[FX(i + 1, j, k)], fy[FY(i, j, k)],
                         fy[FY(i, j + 1, k)], fz[FZ(i, j, k)], fz[FZ(i, j, k + 1)]};
          int m[6] = {across(i - 1, nx, bc[0], 1), across(i + 1, nx, bc[0], 0),
                      across(j - 1, ny, bc[1], 1), across(j + 1, ny, bc[1], 0),
                      across(k - 1, nz, bc[2], 1), across(k + 1, nz, bc[2], 0)};
          size_t nbi[6] = {IDX(m[0], j, k), IDX(m[1], j, k), IDX(i, m[2], k),
                           IDX(i, m[3], k), IDX(i, j, m[4]), IDX(i, j, m[5])};
          double num = 0.0, den = 0.0;
          for (int f = 0; f < 6; ++f) {
            if (m[f] >= 0) {
              num += w[f] * x[nbi[f]];
              den += w[f];
            } else if (m[f] == -1) {
              den += 2.0 * w[f];
            }
          }
          x[IDX(i, j, k)] = (num - h * h * b[IDX(i, j, k)]) / den;
        }
  }
  if (!any_outflow(bc)) oracle_remove_mean(n, x);
  *relres = oracle_residual(nx, ny, nz, h, bc, fx, fy, fz, b, x, r) / bn;
  free(r);
  return status;
}

/* Cell-centred divergence of face velocities (n+1 faces per axis):
 * (div u)_c = sum over axes of (u_high - u_low) / h. */
void oracle_divergence(int nx, int ny, int nz, double h, const double *ux, const double *uy,
                       const double *uz, double *div) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        div[IDX(i, j, k)] = (ux[FX(i + 1, j, k)] - ux[FX(i, j, k)] + uy[FY(i, j + 1, k)] -
                             uy[FY(i, j, k)] + uz[FZ(i, j, k + 1)] - uz[FZ(i, j, k)]) / h;
}

/*
 * Velocity correction of the projection step (Delta t = 1):
 *   u_f = u*_f - beta_f (p_b - p_a - [p]_{a->b}) / h
 * on every face between a (low) and b (high); wall faces keep u*.  An
 * outflow boundary face takes the ghost value -p of its cell for the
 * missing side (no jump: the ghost lies in the cell's fluid).
 * Updates ux, uy, uz (n+1 faces per axis) in place.
 */
void oracle_project(int nx, int ny, int nz, double h, const int bc[3], const double *phi,
                    const double *kappa, const double *fx, const double *fy, const double *fz,
                    double sigma, const double *p, double *ux, double *uy, double *uz) {
  const int periodic[3] = {PER(bc, 0), PER(bc, 1), PER(bc, 2)};
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        if ((i == 0 || i == nx) && !periodic[0]) {
          if (i == 0 && DLO(bc, 0)) ux[FX(i, j, k)] -= fx[FX(i, j, k)] * (2.0 * p[IDX(0, j, k)]) / h;
          if (i == nx && DHI(bc, 0))
            ux[FX(i, j, k)] -= fx[FX(i, j, k)] * (-2.0 * p[IDX(nx - 1, j, k)]) / h;
          continue;
        }
        size_t a = IDX(i == 0 ? nx - 1 : i - 1, j, k), b = IDX(i == nx ? 0 : i, j, k);
        double jp = face_jump(phi[a], phi[b], kappa[a], kappa[b], sigma);
        ux[FX(i, j, k)] -= fx[FX(i, j, k)] * (p[b] - p[a] - jp) / h;
      }
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if ((j == 0 || j == ny) && !periodic[1]) {
          if (j == 0 && DLO(bc, 1)) uy[FY(i, j, k)] -= fy[FY(i, j, k)] * (2.0 * p[IDX(i, 0, k)]) / h;
          if (j == ny && DHI(bc, 1))
            uy[FY(i, j, k)] -= fy[FY(i, j, k)] * (-2.0 * p[IDX(i, ny - 1, k)]) / h;
          continue;
        }
        size_t a = IDX(i, j == 0 ? ny - 1 : j - 1, k), b = IDX(i, j == ny ? 0 : j, k);
        double jp = face_jump(phi[a], phi[b], kappa[a], kappa[b], sigma);
        uy[FY(i, j, k)] -= fy[FY(i, j, k)] * (p[b] - p[a] - jp) / h;
      }
#pragma omp parallel for schedule(static)
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if ((k == 0 || k == nz) && !periodic[2]) {
          if (k == 0 && DLO(bc, 2)) uz[FZ(i, j, k)] -= fz[FZ(i, j, k)] * (2.0 * p[IDX(i, j, 0)]) / h;
          if (k == nz && DHI(bc, 2))
            uz[FZ(i, j, k)] -= fz[FZ(i, j, k)] * (-2.0 * p[IDX(i, j, nz - 1)]) / h;
          continue;
        }
        size_t a = IDX(i, j, k == 0 ? nz - 1 : k - 1), b = IDX(i, j, k == nz ? 0 : k);
        double jp = face_jump(phi[a], phi[b], kappa[a], kappa[b], sigma);
        uz[FZ(i, j, k)] -= fz[FZ(i, j, k)] * (p[b] - p[a] - jp) / h;
      }
}
