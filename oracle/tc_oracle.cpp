// C entry points of the oracle shared library (TEST INFRASTRUCTURE ONLY; see
// tc_oracle.hpp).  Called from Python through ctypes by tests/, the smoke check and
// bench.py's CPU-baseline leg.  All arrays are host arrays of length ncell.
#include "tc_oracle.hpp"
#include "tc_opcount.hpp"

#include <omp.h>
#include <cstring>

namespace oracle {
thread_local OpCount g_ops = {0, 0, 0, 0, 0, 0, 0, 0};
}

using namespace oracle;

extern "C" {
typedef struct {
  const double *n, *chi_pe, *chi_lw, *f_h2, *f_c, *F_lyc, *xi, *Zg, *Zd;
  double *T, *xH2, *xHp;           // in/out
  double *xe, *xCp, *xCO;          // optional out (may be NULL)
  int *nsub, *status, *newton_iters;  // optional out (may be NULL)
} oracle_fields;
}  // extern "C"

static CellIn cell_at(const oracle_fields* f, long long i) {
  CellIn c;
  c.n = f->n[i]; c.chi_pe = f->chi_pe[i]; c.chi_lw = f->chi_lw[i]; c.f_h2 = f->f_h2[i]; c.f_c = f->f_c[i];
  c.F_lyc = f->F_lyc[i]; c.xi = f->xi[i]; c.Zg = f->Zg[i]; c.Zd = f->Zd[i];
  return c;
}

template <class R> static CellOut run_cell(const Params* p, const CellIn& c, double T, double xH2, double xHp,
                                           double dt) {
  return (p->mode == 0) ? step_paper<R>(c, *p, T, xH2, xHp, dt) : step_coupled<R>(c, *p, T, xH2, xHp, dt);
}

static void store(const oracle_fields* f, long long i, const CellOut& o) {
  f->T[i] = o.T; f->xH2[i] = o.xH2; f->xHp[i] = o.xHp;
  if (f->xe) f->xe[i] = o.xe;
  if (f->xCp) f->xCp[i] = o.xCp;
  if (f->xCO) f->xCO[i] = o.xCO;
  if (f->nsub) f->nsub[i] = o.nsub;
  if (f->status) f->status[i] = o.status;
  if (f->newton_iters) f->newton_iters[i] = o.newton_iters;
}

extern "C" {
// Advances ncell cells over dt seconds (one thermochemistry step per cell).
int oracle_step(const Params* p, const oracle_fields* f, long long ncell, double dt, int nthreads) {
  if (!p || !f || ncell < 0) return -1;
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long i = 0; i < ncell; ++i) {
    CellIn c = cell_at(f, i);
    CellOut o = run_cell<double>(p, c, f->T[i], f->xH2[i], f->xHp[i], dt);
    store(f, i, o);
  }
  return 0;
}

// Same as oracle_step but single-threaded under the operation counter; writes the
// summed counts {add, mul, div, sqrt, exp, log, pow, cmp} to counts[8].
int oracle_opcount(const Params* p, const oracle_fields* f, long long ncell, double dt, unsigned long long* counts) {
  if (!p || !f || ncell < 0 || !counts) return -1;
  std::memset(&g_ops, 0, sizeof(g_ops));
  for (long long i = 0; i < ncell; ++i) {
    CellIn c = cell_at(f, i);
    CellOut o = run_cell<Cnt>(p, c, f->T[i], f->xH2[i], f->xHp[i], dt);
    store(f, i, o);
  }
  counts[0] = g_ops.add; counts[1] = g_ops.mul; counts[2] = g_ops.div; counts[3] = g_ops.sqrt;
  counts[4] = g_ops.exp; counts[5] = g_ops.log; counts[6] = g_ops.pow; counts[7] = g_ops.cmp;
  return 0;
}

// Term-by-term evaluation at one state for the unit pins.  cell[9] = {n, chi_pe, chi_lw,
// f_h2, f_c, F_lyc, xi, Zg, Zd}.  Writes ORACLE_NTERMS values in the order listed by
// oracle/__init__.py (TERM_NAMES).  If Td_fixed > 0 it is used as the dust temperature.
#define ORACLE_NTERMS 48
int oracle_terms(const Params* p, const double* cell, double T, double xH2, double xHp, double Td_fixed,
                 double* out) {
  CellIn c{cell[0], cell[1], cell[2], cell[3], cell[4], cell[5], cell[6], cell[7], cell[8]};
  Pre<double> P = prepare<double>(c, *p);
  Equil<double> q = equilibrium(c, P, T, xH2, xHp);
  Source<double> s = source_terms(c, *p, P, T, xH2, xHp, q, Td_fixed);
  double psi = P.G0 * std::sqrt(T) / std::max(q.xe * P.n, 1e-30) + 50.0;
  double v[ORACLE_NTERMS] = {
      q.xe, q.xCp, q.xCO, q.xC, q.xO, q.xOp, q.xMHp,                                   // 0-6
      s.r.kgr, s.r.zcrH2, s.r.zcrH, P.zpd, P.zpiH, P.zpiH2, s.r.zcd, s.r.zci, s.r.arr,  // 7-15
      s.r.agr, s.r.kci, s.r.kcdH, s.r.kcdH2,                                           // 16-19
      s.heat.pe, s.heat.cr, s.heat.pi, s.heat.h2form, s.heat.h2pump, s.heat.h2pd, s.heat.total,  // 20-26
      s.cool.lya, s.cool.ci, s.cool.cd, s.cool.rovib, s.cool.ff, s.cool.rr, s.cool.hyd,         // 27-33
      s.cool.Cp, s.cool.C, s.cool.O, s.cool.CO, s.cool.grrec, s.cool.neb, s.cool.gd, s.cool.cie,  // 34-41
      s.cool.S, s.cool.total, s.Td, s.H, s.CH2, s.CHp};                                 // 42-47
  (void)psi;
  for (int i = 0; i < ORACLE_NTERMS; ++i) out[i] = v[i];
  return ORACLE_NTERMS;
}

// Per-cell constants (for pins on the radiation-derived pieces): writes
// {G0, zpd, zpiH, zpiH2, zpiC_rad, zcrC, lnCO, qH2, Gd, xCtot, xOtot, muH, K}.
int oracle_prepare(const Params* p, const double* cell, double* out) {
  CellIn c{cell[0], cell[1], cell[2], cell[3], cell[4], cell[5], cell[6], cell[7], cell[8]};
  Pre<double> P = prepare<double>(c, *p);
  double v[13] = {P.G0, P.zpd, P.zpiH, P.zpiH2, P.zpiC_rad, P.zcrC, P.lnCO, P.qH2, P.Gd, P.xCtot, P.xOtot, P.muH, P.K};
  for (int i = 0; i < 13; ++i) out[i] = v[i];
  return 13;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Reference time integration for the convergence pin: adaptive Dormand-Prince 5(4)
// on the differential-algebraic system the scheme discretises, dT_mu/dt = H/K,
// dx_s/dt = C_s, with the C/O/e equilibrium and T = mu(x_e, x_H2) T_mu imposed
// consistently at every evaluation (fixed-point iteration on T).
static void dae_rhs(const CellIn& c, const Params& p, const Pre<double>& P, const double* y, double* g,
                    double* Tguess) {
  double T = *Tguess;
  Equil<double> q{};
  for (int k = 0; k < 200; ++k) {
    q = equilibrium(c, P, T, y[1], y[2]);
    double Tn = mu_of(P, q.xe, y[1]) * y[0];
    bool ok = std::fabs(Tn - T) <= 1e-14 * Tn;
    T = Tn;
    if (ok) break;
  }
  q = equilibrium(c, P, T, y[1], y[2]);
  Source<double> s = source_terms(c, p, P, T, y[1], y[2], q, -1.0);
  g[0] = (p.flags & F_FREEZE_T) ? 0.0 : s.H / P.K;
  g[1] = s.CH2;
  g[2] = s.CHp;
  *Tguess = T;
}

extern "C" int oracle_rk45(const Params* p, const double* cell, double T0, double xH20, double xHp0, double dt, double rtol,
                double atol_x, long long max_steps, double* out, long long* nsteps_out) {
  CellIn c{cell[0], cell[1], cell[2], cell[3], cell[4], cell[5], cell[6], cell[7], cell[8]};
  Pre<double> P = prepare<double>(c, *p);
  Equil<double> q = equilibrium(c, P, T0, xH20, xHp0);
  double mu = mu_of(P, q.xe, xH20);
  double y[3] = {T0 / mu, xH20, xHp0};
  double Tg = T0;
  static const double a21 = 1.0 / 5, a31 = 3.0 / 40, a32 = 9.0 / 40, a41 = 44.0 / 45, a42 = -56.0 / 15,
                      a43 = 32.0 / 9, a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561,
                      a54 = -212.0 / 729, a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247,
                      a64 = 49.0 / 176, a65 = -5103.0 / 18656, b1 = 35.0 / 384, b3 = 500.0 / 1113,
                      b4 = 125.0 / 192, b5 = -2187.0 / 6784, b6 = 11.0 / 84, e1 = 71.0 / 57600,
                      e3 = -71.0 / 16695, e4 = 71.0 / 1920, e5 = -17253.0 / 339200, e6 = 22.0 / 525,
                      e7 = -1.0 / 40;
  double t = 0.0, h = dt * 1e-6;
  double k1[3], k2[3], k3[3], k4[3], k5[3], k6[3], k7[3], yt[3], y5[3];
  dae_rhs(c, *p, P, y, k1, &Tg);
  long long steps = 0;
  while (t < dt && steps < max_steps) {
    if (t + h > dt) h = dt - t;
    for (int i = 0; i < 3; ++i) yt[i] = y[i] + h * a21 * k1[i];
    dae_rhs(c, *p, P, yt, k2, &Tg);
    for (int i = 0; i < 3; ++i) yt[i] = y[i] + h * (a31 * k1[i] + a32 * k2[i]);
    dae_rhs(c, *p, P, yt, k3, &Tg);
    for (int i = 0; i < 3; ++i) yt[i] = y[i] + h * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
    dae_rhs(c, *p, P, yt, k4, &Tg);
    for (int i = 0; i < 3; ++i) yt[i] = y[i] + h * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
    dae_rhs(c, *p, P, yt, k5, &Tg);
    for (int i = 0; i < 3; ++i)
      yt[i] = y[i] + h * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
    dae_rhs(c, *p, P, yt, k6, &Tg);
    for (int i = 0; i < 3; ++i) y5[i] = y[i] + h * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
    dae_rhs(c, *p, P, y5, k7, &Tg);
    double err = 0.0;
    for (int i = 0; i < 3; ++i) {
      double ei = h * (e1 * k1[i] + e3 * k3[i] + e4 * k4[i] + e5 * k5[i] + e6 * k6[i] + e7 * k7[i]);
      double sc = (i == 0) ? rtol * std::max(std::fabs(y[i]), std::fabs(y5[i]))
                           : atol_x + rtol * std::max(std::fabs(y[i]), std::fabs(y5[i]));
      err = std::max(err, std::fabs(ei) / sc);
    }
    bool neg = (y5[0] <= 0.0 || y5[1] < 0.0 || y5[2] < 0.0 || !std::isfinite(err));
    if (err <= 1.0 && !neg) {
      t += h;
      for (int i = 0; i < 3; ++i) { y[i] = y5[i]; k1[i] = k7[i]; }
      ++steps;
    }
    double fac = neg ? 0.2 : ((err > 0.0) ? 0.9 * std::pow(err, -0.2) : 5.0);
    fac = std::min(5.0, std::max(0.2, fac));
    h *= fac;
  }
  // Final consistent temperature.
  double g[3];
  dae_rhs(c, *p, P, y, g, &Tg);
  out[0] = Tg; out[1] = y[1]; out[2] = y[2];
  if (nsteps_out) *nsteps_out = steps;
  return (t >= dt) ? 0 : -2;
}
