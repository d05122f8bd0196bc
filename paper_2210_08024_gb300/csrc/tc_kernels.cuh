// Step kernels: one persistent, flattened per-lane loop.
//
// Every lane owns one cell at a time and advances it one substep per loop trip; when
// its cell reaches dt it stores the result and claims the next cell index from a
// warp-aggregated atomic work queue.  All lanes of a warp run the same substep code
// together whatever substep their own cell is at, so cells needing 1 substep and
// cells needing 500 share a warp without idling (Sec. 6.1 subcycling is per cell).
// There is no inter-block wait of any kind: a block exits when the queue is empty.
//
// MODE 0: the paper's sequential update (Sec. 6.1), FP64.
// MODE 1: coupled backward Euler on (T_mu, x_H2, x_H+) by Newton, FP64.
// MODE 2: as 1 with the source terms in FP32 and the Newton update in FP64.
#pragma once
#include <type_traits>

#include "tc_phys.cuh"

namespace tcg {

struct DevFields {
  const double *n, *chi_pe, *chi_lw, *fh2, *fc, *Flyc, *xi, *Zg, *Zd;
  double *T, *xH2, *xHp, *xe, *xCp, *xCO;
  int *nsub, *status;
  long long ncell;
  double Zg_val, Zd_val;
};

// Box table for batched launches: cells [start[b], start[b+1]) belong to box b.
constexpr int MAX_BOX = 64;
struct BoxTable {
  int nbox;
  long long start[MAX_BOX + 1];
  DevFields box[MAX_BOX];
};

constexpr int ST_MAX_SUB = 1, ST_NEWTON = 2, ST_NONFIN = 4;

__device__ __forceinline__ long long claim_cells(unsigned long long* cursor) {
  unsigned mask = __activemask();
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return (long long)base + __popc(mask & ((1u << lane) - 1u));
}

// Lane-resident state of the cell being advanced.
struct LaneState {
  double t, Tmu, xH2, xHp, mu;
  double xe, xCp, xCO, Td;
  int nsub, status;
};

TCG_FN void load_cell(const DevFields& f, long long i, const DevParams& p, CellC<double>& c,
                                          double& T0, double& xH20, double& xHp0) {
  double Zg = f.Zg ? f.Zg[i] : f.Zg_val;
  double Zd = f.Zd ? f.Zd[i] : f.Zd_val;
  double fc = f.fc ? f.fc[i] : 1.0;
  double Fl = f.Flyc ? f.Flyc[i] : 0.0;
  c = make_cell(f.n[i], f.chi_pe[i], f.chi_lw[i], f.fh2[i], fc, Fl, f.xi[i], Zg, Zd, p);
  T0 = f.T[i];
  xH20 = f.xH2[i];
  xHp0 = f.xHp[i];
}

TCG_FN void store_cell(const DevFields& f, long long i, const LaneState& s) {
  f.T[i] = s.mu * s.Tmu;
  f.xH2[i] = s.xH2;
  f.xHp[i] = s.xHp;
  if (f.xe) f.xe[i] = s.xe;
  if (f.xCp) f.xCp[i] = s.xCp;
  if (f.xCO) f.xCO[i] = s.xCO;
  if (f.nsub) f.nsub[i] = s.nsub;
  if (f.status) f.status[i] = s.status;
}

TCG_FN bool finite3(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// Substep length rule of Sec. 6.1 truncated to the remaining time.
TCG_FN double substep_len(const DevParams& p, double rem, double e, double H, double C1, double C2,
                                              bool& last) {
  double d = rem;
  double aH = fabs(H), a1 = fabs(C1), a2 = fabs(C2);
  if (aH > 0.0) d = fmin(d, p.limiter * e / aH);
  if (a1 > 0.0) d = fmin(d, p.limiter / a1);
  if (a2 > 0.0) d = fmin(d, p.limiter / a2);
  last = !(d < rem);
  return last ? rem : d;
}

// ------------------------------------------------------------------ mode 0: paper scheme
TCG_FN void substep_paper(const CellC<double>& c, const DevParams& p, double dt, LaneState& s) {
  const double T = s.mu * s.Tmu;
  const double e = c.K * s.Tmu;
  double H0 = 0.0, CH2 = 0.0, CHp = 0.0, Td0 = -1.0, Hp = 0.0;
  // pass 0: source terms at T (dust temperature solved); pass 1: at T_mu (1 + fd) with
  // every abundance, mu and T_d frozen, for the forward difference dH/dT_mu.
  for (int pass = 0; pass < 2; ++pass) {
    double Tev = T;
    double Tdf = -1.0;
    if (pass == 1) {
      if (H0 == 0.0) break;
      Tev = s.mu * (s.Tmu + p.fd_rel * s.Tmu);
      Tdf = Td0;
    }
    ChemT<double> b = chem_T(c, Tev, p.flags);
    CoolT<double> k = cool_T(c, b, p.flags);
    Equil<double> q;
    q.xe = s.xe; q.xCp = s.xCp; q.xCO = s.xCO;
    q.xOp = c.xOtot * s.xHp;
    q.xC = c.xCtot - s.xCp - s.xCO;
    q.xO = c.xOtot - s.xCO - q.xOp;
    Src<double> sr = source(c, b, k, s.xH2, s.xHp, q, Tdf, s.Td);
    if (pass == 0) { H0 = sr.H; CH2 = sr.CH2; CHp = sr.CHp; Td0 = sr.Td; }
    else Hp = sr.H;
  }
  s.Td = Td0;
  bool last;
  const double dts = substep_len(p, dt - s.t, e, H0, CH2, CHp, last);
  double Tmu_new = s.Tmu;
  if (H0 != 0.0) {
    const double dTmu = p.fd_rel * s.Tmu;
    const double D = (Hp - H0) / dTmu;
    const double tcool = -e / H0;
    const double r = dts / tcool;
    double den = 1.0 + r * (s.Tmu / H0) * D;
    if (den < 0.1) den = 1.0;
    Tmu_new = s.Tmu * (1.0 + (-r) / den);
    const double fl = p.T_floor / s.mu;
    if (Tmu_new < fl) Tmu_new = fl;
  }
  // abundances: 2x2 backward Euler with rates at T^{n+1} = mu^n T_mu^{n+1}, x^n, x_e^n
  const double T1 = s.mu * Tmu_new;
  ChemT<double> b1 = chem_T(c, T1, p.flags);
  HRate<double> r = h_rates(c, b1, s.xH2, s.xHp, s.xe, log_psi(c, b1, s.xe));
  // (I - A dts) X' = X + b dts in closed form, expanded so that every term is
  // non-negative: a = 2 k_gr n + D_H2 and c = I + R are the diagonal loss rates.
  const double a = 2.0 * r.kn + r.DH2;
  const double cc = r.I + r.Rr;
  const double det = 1.0 + (a + cc) * dts + (2.0 * r.kn * r.Rr + r.DH2 * cc) * dts * dts;
  const double n2 = s.xH2 * (1.0 + cc * dts) + r.kn * dts * ((1.0 - s.xHp) + r.Rr * dts);
  const double np = s.xHp * (1.0 + a * dts) + r.I * dts * ((1.0 - 2.0 * s.xH2) + r.DH2 * dts);
  s.xH2 = n2 / det;
  s.xHp = np / det;
  s.Tmu = Tmu_new;
  Equil<double> q = equilibrium(c, b1, s.xH2, s.xHp, s.xe);
  s.xe = q.xe; s.xCp = q.xCp; s.xCO = q.xCO;
  s.mu = c.muH / (1.1 + q.xe - s.xH2);
  s.nsub += 1;
  s.t = last ? dt : s.t + dts;
}

// ------------------------------------------------------------------ modes 1/2: coupled Newton
// f(y) = (H/K, C_H2, C_H+) at T = mu^n y0 with the C/O/e equilibrium and T_d re-solved.
template <class F> TCG_FN void feval(const CellC<F>& c, const ChemT<F>& b, const CoolT<F>& k,
                                                         double y1, double y2, double Kinv, F& xe_guess, F& td_guess,
                                                         double* f) {
  Equil<F> q = equilibrium(c, b, F(y1), F(y2), xe_guess);
  Src<F> s = source(c, b, k, F(y1), F(y2), q, F(-1), td_guess);
  xe_guess = q.xe;
  td_guess = s.Td;
  f[0] = double(s.H) * Kinv;
  f[1] = double(s.CH2);
  f[2] = double(s.CHp);
}

TCG_FN bool solve3(double J[3][3], double b[3], double d[3]) {
  for (int kk = 0; kk < 3; ++kk) {
    int piv = kk;
    double best = fabs(J[kk][kk]);
    for (int i = kk + 1; i < 3; ++i) {
      double v = fabs(J[i][kk]);
      if (v > best) { best = v; piv = i; }
    }
    if (!(best > 0.0)) return false;
    if (piv != kk) {
      for (int j = 0; j < 3; ++j) { double tt = J[kk][j]; J[kk][j] = J[piv][j]; J[piv][j] = tt; }
      double tb = b[kk]; b[kk] = b[piv]; b[piv] = tb;
    }
    for (int i = kk + 1; i < 3; ++i) {
      double m = J[i][kk] / J[kk][kk];
      for (int j = kk; j < 3; ++j) J[i][j] -= m * J[kk][j];
      b[i] -= m * b[kk];
    }
  }
  for (int i = 2; i >= 0; --i) {
    double acc = b[i];
    for (int j = i + 1; j < 3; ++j) acc -= J[i][j] * d[j];
    d[i] = acc / J[i][i];
  }
  return true;
}

// One Newton solve of y - y^n - dts f(y) = 0 from `y` (seed on entry, root on exit).
// Returns iterations used, or -1.
template <class F> TCG_FN int newton_solve(const CellC<F>& c, const DevParams& p, double mu,
                                                               double Kinv, const double* yn, double dts, double* y,
                                                               F& xe_g, F& td_g) {
  const bool fp32 = sizeof(F) == 4;
  const double rtol = fp32 ? p.rtol_mixed : p.rtol;
  const double hrel = fp32 ? 3e-4 : 1e-7;
  const double hfloor = fp32 ? 1e-12 : 1e-17;
  double prev_rel = 1e300;
  for (int it = 1; it <= p.newton_max; ++it) {
    double f0[3], J[3][3];
    ChemT<F> b = chem_T(c, F(mu * y[0]), p.flags);
    CoolT<F> k = cool_T(c, b, p.flags);
    // evaluation order: x_H2 column, x_H+ column, base point (all at the base T), then
    // the T_mu column, so the temperature blocks are built twice per iteration.
    double fx[2][3];
#pragma unroll 1
    for (int j = 1; j < 3; ++j) {
      double h = fmax(hrel * fabs(y[j]), hfloor);
      double y1 = y[1] + ((j == 1) ? h : 0.0), y2 = y[2] + ((j == 2) ? h : 0.0);
      F xg = xe_g, tg = td_g;
      feval<F>(c, b, k, y1, y2, Kinv, xg, tg, fx[j - 1]);
    }
    feval<F>(c, b, k, y[1], y[2], Kinv, xe_g, td_g, f0);
    for (int j = 1; j < 3; ++j) {
      double h = fmax(hrel * fabs(y[j]), hfloor);
      for (int i = 0; i < 3; ++i) J[i][j] = ((i == j) ? 1.0 : 0.0) - dts * (fx[j - 1][i] - f0[i]) / h;
    }
    {
      double h = hrel * y[0];
      ChemT<F> bT = chem_T(c, F(mu * (y[0] + h)), p.flags);
      CoolT<F> kT = cool_T(c, bT, p.flags);
      F xg = xe_g, tg = td_g;
      double fT[3];
      feval<F>(c, bT, kT, y[1], y[2], Kinv, xg, tg, fT);
      for (int i = 0; i < 3; ++i) J[i][0] = ((i == 0) ? 1.0 : 0.0) - dts * (fT[i] - f0[i]) / h;
    }
    double rhs[3], d[3];
    for (int i = 0; i < 3; ++i) rhs[i] = -(y[i] - yn[i] - dts * f0[i]);
    if (!solve3(J, rhs, d)) return -1;
    double lam = 1.0;
    for (int i = 0; i < 3; ++i)
      if (d[i] < 0.0) lam = fmin(lam, 0.99 * y[i] / (-d[i]));
    const double xH = 1.0 - 2.0 * y[1] - y[2];
    const double dxH = -2.0 * d[1] - d[2];
    if (dxH < 0.0) lam = fmin(lam, 0.99 * fmax(xH, 0.0) / (-dxH));
    bool conv = !(lam < 1.0);
    double relmax = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double st = lam * d[i];
      y[i] += st;
      if (fp32) {
        // FP32 source terms put a rounding floor under the step: measure abundances
        // against 1e-10 (the mixed accuracy target is absolute) and stop either at the
        // tolerance or once the step stagnates at the floor.
        relmax = fmax(relmax, fabs(st) / fmax(fabs(y[i]), (i == 0) ? 0.0 : 1e-10));
      } else {
        const double tol = rtol * fabs(y[i]) + 1e-300;
        if (fabs(st) > tol) conv = false;
      }
    }
    if (!finite3(y[0], y[1], y[2])) return -1;
    if (fp32) {
      conv = conv && (relmax <= rtol || (it >= 2 && relmax <= 1e-4 && relmax >= 0.25 * prev_rel));
      prev_rel = relmax;
    }
    if (conv) return it;
  }
  return -1;
}

template <class F>
TCG_FN void substep_newton(const CellC<double>& c, const CellC<F>& cf, const DevParams& p, double dt,
                                               LaneState& s, F& xe_g, F& td_g) {
  // substep length from the source terms at the current state (stored equilibrium)
  const double T = s.mu * s.Tmu;
  const double e = c.K * s.Tmu;
  double H0, CH2, CHp;
  {
    ChemT<F> b = chem_T(cf, F(T), p.flags);
    CoolT<F> k = cool_T(cf, b, p.flags);
    Equil<F> q;
    q.xe = F(s.xe); q.xCp = F(s.xCp); q.xCO = F(s.xCO);
    q.xOp = cf.xOtot * F(s.xHp);
    q.xC = cf.xCtot - q.xCp - q.xCO;
    q.xO = cf.xOtot - q.xCO - q.xOp;
    Src<F> sr = source(cf, b, k, F(s.xH2), F(s.xHp), q, F(-1), td_g);
    td_g = sr.Td;
    H0 = double(sr.H); CH2 = double(sr.CH2); CHp = double(sr.CHp);
  }
  bool last;
  double dts = substep_len(p, dt - s.t, e, H0, CH2, CHp, last);
  const double yn[3] = {s.Tmu, s.xH2, s.xHp};
  const double Kinv = 1.0 / c.K;
  double y[3] = {yn[0], yn[1], yn[2]};
  int it = newton_solve<F>(cf, p, s.mu, Kinv, yn, dts, y, xe_g, td_g);
  int halv = 0;
  while (it < 0 && halv < 30) {
    s.status |= ST_NEWTON;
    dts *= 0.5;
    last = false;
    ++halv;
    y[0] = yn[0]; y[1] = yn[1]; y[2] = yn[2];
    it = newton_solve<F>(cf, p, s.mu, Kinv, yn, dts, y, xe_g, td_g);
  }
  if (it < 0) {
    s.status |= ST_NONFIN;
    s.t = dt;
    return;
  }
  s.nsub += 1;
  s.Tmu = fmax(y[0], p.T_floor / s.mu);
  s.xH2 = y[1];
  s.xHp = y[2];
  // C/O/e equilibrium at the new state and new mu (FP64 in both precisions: it sets mu)
  ChemT<double> b1 = chem_T(c, s.mu * s.Tmu, p.flags);
  Equil<double> q = equilibrium(c, b1, s.xH2, s.xHp, s.xe);
  s.xe = q.xe; s.xCp = q.xCp; s.xCO = q.xCO;
  s.mu = c.muH / (1.1 + q.xe - s.xH2);
  s.t = last ? dt : s.t + dts;
}

// ------------------------------------------------------------------ the kernel
template <int MODE, bool BATCH>
__global__ void __launch_bounds__(128) k_step(DevFields f1, const BoxTable* __restrict__ boxes, DevParams p,
                                               double dt, unsigned long long* cursor, long long ntotal) {
  using F = typename std::conditional<MODE == 2, float, double>::type;
  LaneState s;
  CellC<double> c;
  CellC<float> cf;   // FP32 copy of the cell constants (mixed mode only)
  F xe_g = F(-1), td_g = F(-1);
  DevFields fb;
  long long li = -1;   // local cell index within its box
  bool have = false;
  while (true) {
    if (!have) {
      long long gi = claim_cells(cursor);
      if (gi >= ntotal) break;
      if (BATCH) {
        int lo = 0, hi = boxes->nbox - 1;
        while (lo < hi) {  // last box with start <= gi
          int mid = (lo + hi + 1) >> 1;
          if (boxes->start[mid] <= gi) lo = mid; else hi = mid - 1;
        }
        fb = boxes->box[lo];
        li = gi - boxes->start[lo];
      } else {
        fb = f1;
        li = gi;
      }
      double T0, x20, xp0;
      load_cell(fb, li, p, c, T0, x20, xp0);
      if constexpr (MODE == 2) cf = cast_cell<float>(c);
      ChemT<double> b0 = chem_T(c, T0, p.flags);
      Equil<double> q0 = equilibrium(c, b0, x20, xp0, -1.0);
      s.t = 0.0;
      s.xH2 = x20; s.xHp = xp0;
      s.xe = q0.xe; s.xCp = q0.xCp; s.xCO = q0.xCO;
      s.mu = c.muH / (1.1 + q0.xe - x20);
      s.Tmu = T0 / s.mu;
      s.Td = -1.0;
      s.nsub = 0;
      s.status = 0;
      xe_g = F(q0.xe);
      td_g = F(-1);
      have = true;
    }
    if (s.t < dt) {
      if (s.nsub >= p.max_sub) {
        s.status |= ST_MAX_SUB;
        s.t = dt;
      } else if constexpr (MODE == 0) {
        substep_paper(c, p, dt, s);
      } else if constexpr (MODE == 1) {
        substep_newton<double>(c, c, p, dt, s, xe_g, td_g);
      } else {
        substep_newton<float>(c, cf, p, dt, s, xe_g, td_g);
      }
      if (!finite3(s.Tmu, s.xH2, s.xHp)) {
        s.status |= ST_NONFIN;
        s.t = dt;
      }
    }
    if (!(s.t < dt)) {
      store_cell(fb, li, s);
      have = false;
    }
  }
}

}  // namespace tcg
