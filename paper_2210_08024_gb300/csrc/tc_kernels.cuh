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
// MODE 3: as 2, each Newton solve started from the seed network's prediction.
// MODE 4: as 1, each Newton solve started from the seed network's prediction.
// MODE 2: as 1 with the rates, the C/O/e equilibrium and the heating/cooling sums in
//         FP32, and the Newton update, its residual and the closure
//         x_H = 1 - 2 x_H2 - x_H+ in FP64; a substep whose mixed solve does not
//         converge is re-solved by the FP64 Newton of mode 1 on the same substep.
#pragma once
#include <type_traits>

#include "tc_mlp.cuh"
#include "tc_mlp_mma.cuh"
#include "tc_phys.cuh"

namespace tcg {

struct DevFields {
  const double *n, *chi_pe, *chi_lw, *fh2, *fc, *Flyc, *xi, *Zg, *Zd;
  double *T, *xH2, *xHp, *xe, *xCp, *xCO;
  int *nsub, *status, *iters;
  long long ncell;
  double Zg_val, Zd_val;
  const double* chi0 = nullptr;   // optional per-cell unattenuated FUV scale (driver runs)
  const int* hint = nullptr;      // optional per-cell cost hint for the cost-ordered queue
};

// Box table for batched launches: cells [start[b], start[b+1]) belong to box b.
constexpr int MAX_BOX = 64;
struct BoxTable {
  int nbox;
  long long start[MAX_BOX + 1];
  DevFields box[MAX_BOX];
};

constexpr int ST_MAX_SUB = 1, ST_NEWTON = 2, ST_NONFIN = 4, ST_FALLBACK = 8, ST_POLISH = 16, ST_PREDICTOR = 32;
// seeded modes (informational): a substep's solve started from the seed network's
// prediction converged (ST_SEEDED), or failed and restarted from the start state
// (ST_SEED_FAIL)
constexpr int ST_SEEDED = 64, ST_SEED_FAIL = 128;

__device__ __forceinline__ long long claim_cells(unsigned long long* cursor) {
  unsigned mask = __activemask();
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return (long long)base + __popc(mask & ((1u << lane) - 1u));
}

// Several lanes per cell (LPC = 4, the warp-cooperative kernels): a cell is owned by LPC
// consecutive lanes that hold identical copies of its state and run the same control
// flow; they split the independent function evaluations of a Newton iteration and
// exchange the results by shuffles over the cell's lane mask.  Every lane then forms the
// same Jacobian and takes the same step, so the copies stay identical.
template <int LPC>
TCG_FN int lane_in_cell() {
#ifdef __CUDA_ARCH__
  return (int)(threadIdx.x & (unsigned)(LPC - 1));
#else
  return 0;
#endif
}

// Value of v held by lane r of this lane's cell.
template <int LPC>
TCG_FN double from_lane(double v, int r) {
#ifdef __CUDA_ARCH__
  const unsigned lane = threadIdx.x & 31u;
  const unsigned base = lane & ~(unsigned)(LPC - 1);
  const unsigned mask = ((1u << LPC) - 1u) << base;
  return __shfl_sync(mask, v, (int)(base + (unsigned)r));
#else
  return v;
#endif
}
template <int LPC>
TCG_FN float from_lane(float v, int r) {
#ifdef __CUDA_ARCH__
  const unsigned lane = threadIdx.x & 31u;
  const unsigned base = lane & ~(unsigned)(LPC - 1);
  const unsigned mask = ((1u << LPC) - 1u) << base;
  return __shfl_sync(mask, v, (int)(base + (unsigned)r));
#else
  return v;
#endif
}

// Work-queue claim for cells of LPC lanes: the first lane of the cell takes the next
// index and hands it to the others by a shuffle over the cell's explicit lane mask
// (__activemask could return part of a cell whose lanes are briefly apart, so the
// claim does not aggregate over the warp).
template <int LPC>
__device__ __forceinline__ long long claim_cells_lpc(unsigned long long* cursor) {
  if constexpr (LPC == 1) {
    return claim_cells(cursor);
  } else {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned base = lane & ~(unsigned)(LPC - 1);
    const unsigned mask = ((1u << LPC) - 1u) << base;
    unsigned long long v = 0;
    if (lane == base) v = atomicAdd(cursor, 1ull);
    v = __shfl_sync(mask, v, (int)base);
    return (long long)v;
  }
}

// Lane-resident state of the cell being advanced.
struct LaneState {
  double t, Tmu, xH2, xHp, mu;
  double xe, xCp, xCO, Td;
  int nsub, status, iters;
};

TCG_FN void load_cell(const DevFields& f, long long i, const DevParams& p, CellC<double>& c,
                                          double& T0, double& xH20, double& xHp0) {
  double Zg = f.Zg ? f.Zg[i] : f.Zg_val;
  double Zd = f.Zd ? f.Zd[i] : f.Zd_val;
  double fc = f.fc ? f.fc[i] : 1.0;
  double Fl = f.Flyc ? f.Flyc[i] : 0.0;
  c = make_cell(f.n[i], f.chi_pe[i], f.chi_lw[i], f.fh2[i], fc, Fl, f.xi[i], Zg, Zd, p, f.chi0 ? f.chi0[i] : -1.0);
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
  if (f.iters) f.iters[i] = s.iters;
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
  TCG_COUNT_D(substep_paper);
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
    q.lpsi = log_psi(c, b, q.xe);
    Src<double> sr = source(c, b, k, s.xH2, s.xHp, 1.0 - 2.0 * s.xH2 - s.xHp, q, Tdf, s.Td);
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
  HRate<double> r = h_rates(c, b1, s.xH2, 1.0 - 2.0 * s.xH2 - s.xHp, s.xe, log_psi(c, b1, s.xe));
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

// ------------------------------------------------------------------ mode 1: coupled Newton, FP64
// f(y) = (H/K, C_H2, C_H+) at T = mu^n y0 with the C/O/e equilibrium and T_d re-solved,
// the source terms in precision F (double: the FP64 solves; df64: the high-precision
// evaluations of the mixed solve), the state and f in FP64.  `qout`, when given,
// receives the C/O/e equilibrium of the evaluation.
template <class F>
TCG_FN void feval_t(const CellC<F>& c, const ChemT<F>& b, const CoolT<F>& k, double y1, double y2, double Kinv,
                    F& xe_guess, F& td_guess, double* f, Equil<F>* qout = nullptr, int eq_newton_max = 100) {
  const F fy1 = to_prec<F>(y1), fy2 = to_prec<F>(y2);
  Equil<F> q = equilibrium(c, b, fy1, fy2, xe_guess, eq_newton_max);
  if (qout) *qout = q;
  Src<F> s = source(c, b, k, fy1, fy2, to_prec<F>(1.0 - 2.0 * y1 - y2), q, F(-1.0), td_guess);
  xe_guess = q.xe;
  td_guess = s.Td;
  f[0] = double(s.H) * Kinv;
  f[1] = double(s.CH2);
  f[2] = double(s.CHp);
}
TCG_FN void feval64(const CellC<double>& c, const ChemT<double>& b, const CoolT<double>& k, double y1,
                    double y2, double Kinv, double& xe_guess, double& td_guess, double* f,
                    Equil<double>* qout = nullptr, int eq_newton_max = 100) {
  feval_t<double>(c, b, k, y1, y2, Kinv, xe_guess, td_guess, f, qout, eq_newton_max);
}

// The FP64 fields of a C/O/e equilibrium solved in precision F.
template <class F>
TCG_FN Equil<double> equil64(const Equil<F>& q) {
  Equil<double> r;
  r.xe = double(q.xe); r.xCp = double(q.xCp); r.xCO = double(q.xCO); r.xC = double(q.xC);
  r.xO = double(q.xO); r.xOp = double(q.xOp); r.xMHp = double(q.xMHp); r.lpsi = double(q.lpsi);
  return r;
}

// Gaussian elimination with partial pivoting on a 3x3 system, in the precision F of its
// operands (FP64 for the Newton steps of the FP64 solves; FP32 for the corrections of
// the mixed solve, whose Jacobian is an FP32 forward difference good to ~1e-3 anyway).
template <class F>
TCG_FN bool solve3(F J[3][3], F b[3], F d[3]) {
  for (int kk = 0; kk < 3; ++kk) {
    int piv = kk;
    F best = m_abs(J[kk][kk]);
    for (int i = kk + 1; i < 3; ++i) {
      F v = m_abs(J[i][kk]);
      if (v > best) { best = v; piv = i; }
    }
    if (!(best > F(0))) return false;
    if (piv != kk) {
      for (int j = 0; j < 3; ++j) { F tt = J[kk][j]; J[kk][j] = J[piv][j]; J[piv][j] = tt; }
      F tb = b[kk]; b[kk] = b[piv]; b[piv] = tb;
    }
    for (int i = kk + 1; i < 3; ++i) {
      F m = J[i][kk] / J[kk][kk];
      for (int j = kk; j < 3; ++j) J[i][j] -= m * J[kk][j];
      b[i] -= m * b[kk];
    }
  }
  for (int i = 2; i >= 0; --i) {
    F acc = b[i];
    for (int j = i + 1; j < 3; ++j) acc -= J[i][j] * d[j];
    d[i] = acc / J[i][i];
  }
  return true;
}

// Damping of a Newton step d, by blocks (the root is unchanged, only the path to it):
// T_mu takes the step length lamT that keeps it at >= 1% of its value; x_H2 and x_H+
// share a length lamX that keeps them and x_H = 1 - 2 x_H2 - x_H+ at >= 1% of their
// values (fraction 0.99 to the boundary), so that neither block freezes the other.  If
// the x_H bound alone would cut the abundance step below 1% of its length, the step is
// projected onto that bound instead (the smallest change along its normal (-2, -1)),
// so the iteration slides along it rather than stalling.  An abundance whose step is
// below 1e-8 in absolute terms does not limit lamX and is kept at >= 1% of its value on
// its own.  Applies the step to y, writes the steps taken to st and returns true if no
// limit acted (a full Newton step).
TCG_FN bool damped_step(double* y, const double* d, double* st) {
  double lamT = 1.0, lamX = 1.0;
  if (d[0] < 0.0) lamT = fmin(lamT, 0.99 * y[0] / (-d[0]));
  bool tiny[3] = {false, false, false};
  for (int i = 1; i < 3; ++i) {
    tiny[i] = !(fabs(d[i]) > 1e-8);
    if (d[i] < 0.0 && !tiny[i]) lamX = fmin(lamX, 0.99 * y[i] / (-d[i]));
  }
  const double xH = 1.0 - 2.0 * y[1] - y[2];
  const double dxH = -2.0 * d[1] - d[2];
  bool proj = false;
  double e1 = d[1], e2 = d[2];
  if (dxH < 0.0) {
    const double cap = 0.99 * fmax(xH, 0.0) / (-dxH);
    if (cap < 0.01) {
      const double lim = -0.99 * fmax(xH, 0.0);
      const double beta = (dxH - lim) / 5.0;
      e1 += 2.0 * beta;
      e2 += beta;
      proj = true;
      lamX = 1.0;
      tiny[1] = !(fabs(e1) > 1e-8);
      tiny[2] = !(fabs(e2) > 1e-8);
      if (e1 < 0.0 && !tiny[1]) lamX = fmin(lamX, 0.99 * y[1] / (-e1));
      if (e2 < 0.0 && !tiny[2]) lamX = fmin(lamX, 0.99 * y[2] / (-e2));
    } else {
      lamX = fmin(lamX, cap);
    }
  }
  const double dd[3] = {d[0], e1, e2};
  bool full = !(lamT < 1.0) && !(lamX < 1.0) && !proj;
  for (int i = 0; i < 3; ++i) {
    double s = ((i == 0) ? lamT : lamX) * dd[i];
    if (tiny[i] && y[i] + s < 0.01 * y[i]) {
      s = -0.99 * y[i];
      full = false;
    }
    const double yi = y[i] + s;
    st[i] = yi - y[i];
    y[i] = yi;
  }
  return full;
}

// Out-of-line forms of the two routines above for the mixed kernels: their hot loop is
// bound by instruction fetch, and inlined at each of their call sites these made the
// mixed step 4% slower (68.2 against 65.3 ms on the 128^3 slab); the FP64 kernels keep
// them inlined (out of line the seeded FP64 step ran 358 against 321 ms).
__host__ __device__ __noinline__ inline bool solve3_ool(float J[3][3], float b[3], float d[3]) {
  return solve3<float>(J, b, d);
}
__host__ __device__ __noinline__ inline bool damped_step_ool(double* y, const double* d, double* st) {
  return damped_step(y, d, st);
}

// Jacobian reuse.  Once a full (undamped) Newton step is below JAC_REUSE |y_i| in every
// component, the next iterations keep that Jacobian (chord iterations: f at the base
// point only, instead of at four points) for as long as each step is full and at most
// half the previous one; otherwise the next iteration rebuilds it.  The root and the
// convergence test are those of the plain iteration: near the root a chord step
// contracts by about JAC_REUSE times the relative curvature of f, far below the 1/2 that
// keeps the reuse going.
constexpr double JAC_REUSE = 1e-3;

// One iteration on y - y^n - dts f(y) = 0.  With `reuse` false: forward-difference
// Jacobian (relative step 1e-7, abundance steps floored at 1e-17), kept in Jk; with
// `reuse` true: the Jacobian Jk of an earlier iteration.  Then a damped step and the
// test that every full step is below rtol |y_i|.  `rel` returns the step's largest
// relative component and `full` whether no damping limit acted.  Returns 1 when
// converged, 0 to continue, -1 on failure (singular Jacobian or a non-finite state).
template <int LPC = 1>
TCG_FN int newton_iter(const CellC<double>& c, const DevParams& p, double mu, double Kinv, const double* yn,
                       double dts, double* y, double& xe_g, double& td_g, double (*Jk)[3], bool reuse,
                       double& rel, bool& full, Equil<double>* qb,
                       const ChemT<double>* b0 = nullptr, const CoolT<double>* k0 = nullptr) {
  double f0[3], J[3][3];
  if constexpr (LPC == 4) {
    if (reuse) {
      TCG_COUNT_D(chord64_it);
      ChemT<double> b = chem_T(c, mu * y[0], p.flags);
      CoolT<double> k = cool_T(c, b, p.flags);
      feval64(c, b, k, y[1], y[2], Kinv, xe_g, td_g, f0, qb);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = Jk[i][j];
    } else {
      TCG_COUNT_D(newton64_it);
      // Warp-cooperative forward-difference Jacobian: lane q of the cell evaluates f at the
      // base point (q = 0) or with x_H2 (q = 1), x_H+ (q = 2) or T_mu (q = 3) perturbed,
      // each from the same x_e and T_d guesses; the four results are exchanged.
      const int q = lane_in_cell<4>();
      const double h0 = 1e-7 * y[0];
      const double h1 = fmax(1e-7 * fabs(y[1]), 1e-17), h2 = fmax(1e-7 * fabs(y[2]), 1e-17);
      double fq[3];
      Equil<double> qq;
      double xg = xe_g, tg = td_g;
      {
        ChemT<double> b = chem_T(c, mu * ((q == 3) ? y[0] + h0 : y[0]), p.flags);
        CoolT<double> k = cool_T(c, b, p.flags);
        feval64(c, b, k, y[1] + ((q == 1) ? h1 : 0.0), y[2] + ((q == 2) ? h2 : 0.0), Kinv, xg, tg, fq, &qq);
      }
      const double s0 = dts / h0, s1 = dts / h1, s2 = dts / h2;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        f0[i] = from_lane<4>(fq[i], 0);
        const double f1 = from_lane<4>(fq[i], 1), f2 = from_lane<4>(fq[i], 2), fT = from_lane<4>(fq[i], 3);
        J[i][1] = ((i == 1) ? 1.0 : 0.0) - s1 * (f1 - f0[i]);
        J[i][2] = ((i == 2) ? 1.0 : 0.0) - s2 * (f2 - f0[i]);
        J[i][0] = ((i == 0) ? 1.0 : 0.0) - s0 * (fT - f0[i]);
      }
      xe_g = from_lane<4>(xg, 0);
      td_g = from_lane<4>(tg, 0);
      if (qb) {
        qb->xe = from_lane<4>(qq.xe, 0);
        qb->xCp = from_lane<4>(qq.xCp, 0);
        qb->xCO = from_lane<4>(qq.xCO, 0);
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Jk[i][j] = J[i][j];
    }
  } else {
    // One lane per cell: the base point is evaluated by every lane of the warp on one
    // path, whether the lane then reuses its Jacobian (chord iteration) or rebuilds it,
    // so a warp whose lanes mix the two runs the base evaluation once, not once per
    // branch.  Rebuild order: base point, x_H2 column, x_H+ column (all at the base T),
    // then the T_mu column from the base point's temperature blocks stepped to T + dT
    // (temp_blocks_step).  The columns start their C/O/e and dust-temperature solves from the base
    // point's roots, ~1e-7 away, and take one Newton step of the C/O/e balance
    // (converged to ~1e-14 from there; the loop would take a second to confirm it).  The
    // temperature blocks at the base point are given by the caller at a substep's first
    // iteration (the substep start's, the same temperature), else built here.
    if (reuse) TCG_COUNT_D(chord64_it);
    else TCG_COUNT_D(newton64_it);
    ChemT<double> b;
    CoolT<double> k;
    if (b0) {
      b = *b0;
      k = *k0;
    } else {
      b = chem_T(c, mu * y[0], p.flags);
      k = cool_T(c, b, p.flags);
    }
    feval64(c, b, k, y[1], y[2], Kinv, xe_g, td_g, f0, qb);
    if (reuse) {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = Jk[i][j];
    } else {
#pragma unroll 1
      for (int j = 1; j < 3; ++j) {
        const double h = fmax(1e-7 * fabs(y[j]), 1e-17);
        const double y1 = y[1] + ((j == 1) ? h : 0.0), y2 = y[2] + ((j == 2) ? h : 0.0);
        double xg = xe_g, tg = td_g, fx[3];
        feval64(c, b, k, y1, y2, Kinv, xg, tg, fx, nullptr, 1);
        const double sj = dts / h;
        for (int i = 0; i < 3; ++i) J[i][j] = ((i == j) ? 1.0 : 0.0) - sj * (fx[i] - f0[i]);
      }
      {
        // the temperature blocks at T + dT stepped from the base point's (first order in
        // dT = 1e-7 T: the same column to the difference's truncation error)
        double h = 1e-7 * y[0];
        ChemT<double> bT;
        CoolT<double> kT;
        temp_blocks_step(c, b, k, mu * (y[0] + h), p.flags, bT, kT);
        double xg = xe_g, tg = td_g;
        double fT[3];
        feval64(c, bT, kT, y[1], y[2], Kinv, xg, tg, fT, nullptr, 1);
        const double s0 = dts / h;
        for (int i = 0; i < 3; ++i) J[i][0] = ((i == 0) ? 1.0 : 0.0) - s0 * (fT[i] - f0[i]);
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Jk[i][j] = J[i][j];
    }
  }
  double rhs[3], d[3];
  for (int i = 0; i < 3; ++i) rhs[i] = -(y[i] - yn[i] - dts * f0[i]);
  if (!solve3<double>(J, rhs, d)) return -1;
  double st[3];
  full = damped_step(y, d, st);
  bool conv = full;
  rel = 0.0;
  for (int i = 0; i < 3; ++i) {
    if (fabs(st[i]) > p.rtol * fabs(y[i]) + 1e-300) conv = false;
    rel = fmax(rel, fabs(st[i]) / (fabs(y[i]) + 1e-300));
  }
  if (!finite3(y[0], y[1], y[2])) return -1;
  return conv ? 1 : 0;
}

// One Newton solve from `y` (seed on entry, root on exit), with the Jacobian reuse
// above.  Returns the iterations used (chord iterations included), or -1.  `qb`, when
// given, receives the C/O/e equilibrium at the last base point, the root's predecessor
// (within 1e-12 relative of the root when the solve converges).
template <int LPC = 1>
TCG_FN int newton_solve(const CellC<double>& c, const DevParams& p, double mu, double Kinv, const double* yn,
                        double dts, double* y, double& xe_g, double& td_g, int maxit = 0,
                        Equil<double>* qb = nullptr, int* spent = nullptr,
                        const ChemT<double>* b0 = nullptr, const CoolT<double>* k0 = nullptr) {
  const int nmax = (maxit > 0) ? maxit : p.newton_max;
  double Jk[3][3];
  bool reuse = false;
  double prev = 1.0;
  for (int it = 1; it <= nmax; ++it) {
    double rel;
    bool full;
    const int r = newton_iter<LPC>(c, p, mu, Kinv, yn, dts, y, xe_g, td_g, Jk, reuse, rel, full, qb,
                                   (it == 1) ? b0 : nullptr, (it == 1) ? k0 : nullptr);
    if (spent) *spent = it;
    if (r < 0) return -1;
    if (r > 0) return it;
    reuse = full && rel < JAC_REUSE && (!reuse || rel <= 0.5 * prev);
    prev = rel;
  }
  return -1;
}

// Source terms at the substep start from the stored equilibrium (x_e, x_C+, x_CO),
// with the dust temperature solved; gives the substep length of Sec. 6.1.
template <class F>
TCG_FN void start_sources(const CellC<F>& cf, const DevParams& p, const LaneState& s, F& td_g, double& H0,
                          double& CH2, double& CHp, ChemT<F>* bo = nullptr, CoolT<F>* ko = nullptr) {
  const double T = s.mu * s.Tmu;
  ChemT<F> b = chem_T(cf, to_prec<F>(T), p.flags);
  CoolT<F> k = cool_T(cf, b, p.flags);
  if (bo) { *bo = b; *ko = k; }
  Equil<F> q;
  q.xe = to_prec<F>(s.xe); q.xCp = to_prec<F>(s.xCp); q.xCO = to_prec<F>(s.xCO);
  q.xOp = cf.xOtot * to_prec<F>(s.xHp);
  q.xC = cf.xCtot - q.xCp - q.xCO;
  q.xO = cf.xOtot - q.xCO - q.xOp;
  q.lpsi = log_psi(cf, b, q.xe);
  Src<F> sr = source(cf, b, k, to_prec<F>(s.xH2), to_prec<F>(s.xHp), to_prec<F>(1.0 - 2.0 * s.xH2 - s.xHp), q, F(-1),
                     td_g);
  td_g = sr.Td;
  const double n = double(cf.n);
  H0 = n * double(sr.G) - n * n * double(sr.L);
  CH2 = double(sr.form) - double(sr.dest);
  CHp = double(sr.ion) - double(sr.rec);
}

// Accepts the substep's root y: applies the temperature floor, re-solves the C/O/e
// equilibrium at the new state in precision F and updates mu.
template <class F>
TCG_FN void finish_substep(const CellC<F>& cf, double muH, const DevParams& p, double dt, double dts, bool last,
                           const double* y, LaneState& s) {
  s.nsub += 1;
  s.Tmu = fmax(y[0], p.T_floor / s.mu);
  s.xH2 = y[1];
  s.xHp = y[2];
  ChemT<F> b1 = chem_T(cf, F(s.mu * s.Tmu), p.flags);
  Equil<F> q = equilibrium(cf, b1, F(s.xH2), F(s.xHp), F(s.xe));
  s.xe = double(q.xe); s.xCp = double(q.xCp); s.xCO = double(q.xCO);
  s.mu = muH / (1.1 + s.xe - s.xH2);
  s.t = last ? dt : s.t + dts;
}

// Accepts the root y of a substep whose last FP64 evaluation of f solved the C/O/e
// equilibrium `q` at the root's predecessor y' (within 1e-12 of y relative for the FP64
// Newton solve, within 1e-8 for the polish of the mixed one): that equilibrium sets
// x_e, x_C+, x_CO and mu for the next substep instead of a new solve at y.  The
// difference is that of the equilibrium between two states that close.  With the temperature floor active the
// equilibrium is solved at the floored state instead.
TCG_FN void finish_substep_q(const CellC<double>& c, const DevParams& p, double dt, double dts, bool last,
                             const double* y, const Equil<double>& q, LaneState& s) {
  if (!(y[0] >= p.T_floor / s.mu)) {
    finish_substep<double>(c, c.muH, p, dt, dts, last, y, s);
    return;
  }
  s.nsub += 1;
  s.Tmu = y[0];
  s.xH2 = y[1];
  s.xHp = y[2];
  s.xe = q.xe; s.xCp = q.xCp; s.xCO = q.xCO;
  s.mu = c.muH / (1.1 + s.xe - s.xH2);
  s.t = last ? dt : s.t + dts;
}

// Start point for a substep whose Newton solve from the start state fails (Sec. 6.1
// gives no solver for the coupled scheme).  In hot gas where H is ionised as fast as H2
// dissociation frees it, the root lies next to x_H = 0 and the Newton direction at the
// start state points far outside the admissible region; the damped iteration stalls in
// the corner x_H -> 0.  Block sweeps on the same backward-Euler equations instead:
// abundances by the paper's closed-form 2x2 backward Euler with every rate at the
// current iterate (non-negative by construction), then T_mu by one Newton step on its
// own equation T_mu - T_mu^n - dts H/K = 0 at those abundances (forward-difference slope,
// relative step 1e-7; the explicit value T_mu^n + dts H/K when the slope is below 0.1),
// kept within a factor 2 of the old value.  Stops when every component changed by less
// than 1e-3 relative (abundances relative to max(x, 1e-6)), or after 50 sweeps.
TCG_FN void picard_predictor(const CellC<double>& c, const DevParams& p, double mu, double Kinv, const double* yn,
                             double dts, double* y, double& xe_g, double& td_g) {
  y[0] = yn[0]; y[1] = yn[1]; y[2] = yn[2];
#pragma unroll 1
  for (int k = 0; k < 50; ++k) {
    TCG_COUNT_D(picard_it);
    ChemT<double> b = chem_T(c, mu * y[0], p.flags);
    const Equil<double> q = equilibrium(c, b, y[1], y[2], xe_g);
    xe_g = q.xe;
    const HRate<double> r = h_rates(c, b, y[1], 1.0 - 2.0 * y[1] - y[2], q.xe, q.lpsi);
    const double a = 2.0 * r.kn + r.DH2;
    const double cc = r.I + r.Rr;
    const double det = 1.0 + (a + cc) * dts + (2.0 * r.kn * r.Rr + r.DH2 * cc) * dts * dts;
    const double x2 = (yn[1] * (1.0 + cc * dts) + r.kn * dts * ((1.0 - yn[2]) + r.Rr * dts)) / det;
    const double xp = (yn[2] * (1.0 + a * dts) + r.I * dts * ((1.0 - 2.0 * yn[1]) + r.DH2 * dts)) / det;
    double fa[3], fb[3];
    {
      CoolT<double> k = cool_T(c, b, p.flags);
      feval64(c, b, k, x2, xp, Kinv, xe_g, td_g, fa);
    }
    const double h = 1e-7 * y[0];
    {
      ChemT<double> bT = chem_T(c, mu * (y[0] + h), p.flags);
      CoolT<double> kT = cool_T(c, bT, p.flags);
      double xg = xe_g, tg = td_g;
      feval64(c, bT, kT, x2, xp, Kinv, xg, tg, fb);
    }
    const double g = y[0] - yn[0] - dts * fa[0];
    const double gp = 1.0 - dts * (fb[0] - fa[0]) / h;
    double Tm = (gp > 0.1) ? y[0] - g / gp : yn[0] + dts * fa[0];
    Tm = fmin(fmax(Tm, 0.5 * y[0]), 2.0 * y[0]);
    double ch = fabs(Tm - y[0]) / y[0];
    ch = fmax(ch, fabs(x2 - y[1]) / fmax(y[1], 1e-6));
    ch = fmax(ch, fabs(xp - y[2]) / fmax(y[2], 1e-6));
    y[0] = Tm; y[1] = x2; y[2] = xp;
    if (!finite3(y[0], y[1], y[2])) return;
    if (ch < 1e-3) return;
  }
}

// Iteration cap of the Newton solve from the predictor, in units of newton_max: in
// thermally unstable substeps the damped iteration can take a few hundred iterations to
// reach the root (measured up to ~300), and the alternative, halving the substep,
// changes the substep grid and with it the result.
constexpr int RESCUE_ITER_FACTOR = 8;

// One substep's FP64 Newton solve at length dts: from the start state (newton_max
// iterations), and if that fails, from the predictor above (flagging ST_PREDICTOR;
// RESCUE_ITER_FACTOR newton_max iterations).  Returns the iterations of the successful
// solve, or -1.
template <int LPC = 1>
TCG_FN int solve_from_start64(const CellC<double>& c, const DevParams& p, double mu, double Kinv, const double* yn,
                              double dts, double* y, double& xe_g, double& td_g, int& status, Equil<double>* qb,
                              const ChemT<double>* b0 = nullptr, const CoolT<double>* k0 = nullptr) {
  y[0] = yn[0]; y[1] = yn[1]; y[2] = yn[2];
  int it = newton_solve<LPC>(c, p, mu, Kinv, yn, dts, y, xe_g, td_g, 0, qb, nullptr, b0, k0);
  if (it >= 0) return it;
  status |= ST_PREDICTOR;
  picard_predictor(c, p, mu, Kinv, yn, dts, y, xe_g, td_g);
  if (!finite3(y[0], y[1], y[2])) return -1;
  return newton_solve<LPC>(c, p, mu, Kinv, yn, dts, y, xe_g, td_g, RESCUE_ITER_FACTOR * p.newton_max, qb);
}

// A seeded Newton solve that has not converged after this many iterations is abandoned
// and the substep restarts from its start state: a poor seed then costs little.
constexpr int SEED_MAXIT = 6;
// Largest predicted changes (log10 T, abundances) for which a seed is used.
constexpr float SEED_MAX_DLOGT = 0.02f, SEED_MAX_DX = 0.02f;

// f(y) from FP32 source terms; the closure x_H and the net sums H = n G - n^2 L,
// C_H2 = form - dest, C_H+ = ion - rec are formed in FP64 from the FP32 parts.
TCG_FN void feval32(const CellC<float>& cf, const ChemT<float>& b, const CoolT<float>& k, double y1, double y2,
                    double Kinv, float& xe_guess, float& td_guess, double* f) {
  const double xH = 1.0 - 2.0 * y1 - y2;
  Equil<float> q = equilibrium(cf, b, float(y1), float(y2), xe_guess);
  Src<float> s = source(cf, b, k, float(y1), float(y2), float(xH), q, -1.f, td_guess);
  xe_guess = q.xe;
  td_guess = s.Td;
  const double n = double(cf.n);
  f[0] = (n * double(s.G) - n * n * double(s.L)) * Kinv;
  f[1] = double(s.form) - double(s.dest);
  f[2] = double(s.ion) - double(s.rec);
}

// FP32 forward-difference Jacobian (relative step 1e-3) of the backward-Euler residual
// at y, built afresh at the FP32 iteration's root before the df64 polish: at the root
// itself it is as good as an FP32 difference gets (~1e-3), so the polish contracts by
// about that much per correction instead of by the error of a Jacobian built several
// iterations earlier.  With LPC = 4 the four evaluations are split over the cell's lanes.
template <int LPC = 1>
TCG_FN void fd_jacobian32(const CellC<float>& cf, const DevParams& p, double mu, double Kinv, double dts,
                          const double* y, float xe_g, float td_g, float J[3][3]) {
  const double h0 = 1e-3 * y[0];
  const double h1 = fmax(1e-3 * fabs(y[1]), 1e-12), h2 = fmax(1e-3 * fabs(y[2]), 1e-12);
  double f0[3], f1[3], f2[3], fT[3];
  if constexpr (LPC == 4) {
    const int q = lane_in_cell<LPC>();
    double fq[3];
    float xg = xe_g, tg = td_g;
    {
      ChemT<float> b = chem_T(cf, float(mu * ((q == 3) ? y[0] + h0 : y[0])), p.flags);
      CoolT<float> k = cool_T(cf, b, p.flags);
      feval32(cf, b, k, y[1] + ((q == 1) ? h1 : 0.0), y[2] + ((q == 2) ? h2 : 0.0), Kinv, xg, tg, fq);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f0[i] = from_lane<LPC>(fq[i], 0);
      f1[i] = from_lane<LPC>(fq[i], 1);
      f2[i] = from_lane<LPC>(fq[i], 2);
      fT[i] = from_lane<LPC>(fq[i], 3);
    }
  } else {
    ChemT<float> b = chem_T(cf, float(mu * y[0]), p.flags);
    CoolT<float> k = cool_T(cf, b, p.flags);
    float xg = xe_g, tg = td_g;
    feval32(cf, b, k, y[1], y[2], Kinv, xg, tg, f0);
    xg = xe_g; tg = td_g;
    feval32(cf, b, k, y[1] + h1, y[2], Kinv, xg, tg, f1);
    xg = xe_g; tg = td_g;
    feval32(cf, b, k, y[1], y[2] + h2, Kinv, xg, tg, f2);
    ChemT<float> bT = chem_T(cf, float(mu * (y[0] + h0)), p.flags);
    CoolT<float> kT = cool_T(cf, bT, p.flags);
    xg = xe_g; tg = td_g;
    feval32(cf, bT, kT, y[1], y[2], Kinv, xg, tg, fT);
  }
  // the differences of f in FP64 (nearby values), the columns in FP32
  const float s0 = float(dts) / float(h0), s1 = float(dts) / float(h1), s2 = float(dts) / float(h2);
  for (int i = 0; i < 3; ++i) {
    J[i][0] = ((i == 0) ? 1.f : 0.f) - s0 * float(fT[i] - f0[i]);
    J[i][1] = ((i == 1) ? 1.f : 0.f) - s1 * float(f1[i] - f0[i]);
    J[i][2] = ((i == 2) ? 1.f : 0.f) - s2 * float(f2[i] - f0[i]);
  }
}

// Seeded FP64 solve (mode 4): FP64 chord iterations from the seed with the FP32
// forward-difference Jacobian built at the seed.  The network puts the seed within
// ~2e-4 of the root, so each iteration contracts by about the Jacobian's error (~1e-3)
// and the FP64 residual brings the iterate to the FP64 root in a few evaluations of f,
// with the convergence test of the FP64 Newton solve (every step below rtol |y_i|).
// Returns the iterations, or -1 if a step fails to contract by half, the state is not
// finite, or SEED_MAXIT + 2 iterations pass; `spent` receives the iterations made.
template <int LPC = 1>
TCG_FN int chord64_from_seed(const CellC<double>& c, const CellC<float>& cf, const DevParams& p, double mu, double Kinv,
                             const double* yn, double dts, double* y, double& xe_g, double& td_g, Equil<double>* qb,
                             int* spent) {
  float J[3][3];
  fd_jacobian32<LPC>(cf, p, mu, Kinv, dts, y, float(xe_g), float(td_g), J);
  double prev = -1.0;
  for (int it = 1; it <= SEED_MAXIT + 2; ++it) {
    TCG_COUNT_D(chord64_it);
    *spent = it;
    ChemT<double> b = chem_T(c, mu * y[0], p.flags);
    CoolT<double> k = cool_T(c, b, p.flags);
    double f0[3];
    feval64(c, b, k, y[1], y[2], Kinv, xe_g, td_g, f0, qb);
    double Jw[3][3], rhs[3], d[3];
    for (int i = 0; i < 3; ++i) {
      rhs[i] = -(y[i] - yn[i] - dts * f0[i]);
      for (int jj = 0; jj < 3; ++jj) Jw[i][jj] = double(J[i][jj]);
    }
    if (!solve3<double>(Jw, rhs, d)) return -1;
    double st[3];
    const bool full = damped_step(y, d, st);
    if (!finite3(y[0], y[1], y[2])) return -1;
    bool conv = full;
    double nrm = 0.0;
    for (int i = 0; i < 3; ++i) {
      if (fabs(st[i]) > p.rtol * fabs(y[i]) + 1e-300) conv = false;
      nrm = fmax(nrm, fabs(st[i]) / (fabs(y[i]) + 1e-300));
    }
    if (conv) return it;
    if (prev > 0.0 && nrm > 0.5 * prev) return -1;
    prev = nrm;
  }
  return -1;
}


// Solves one substep of length dts by the FP64 Newton iteration, from `seed` when
// given (the root is the same; a seeded solve that fails is retried from the start
// state), else from the start state, then from the predictor; a substep that fails
// from both is retried at half length (up to 30 times) and the cell flagged ST_NEWTON.
template <int LPC = 1>
TCG_FN void solve_substep64(const CellC<double>& c, const DevParams& p, double dt, double dts, bool last,
                            LaneState& s, double& xe_g, double& td_g, const double* seed = nullptr,
                            const CellC<float>* cf = nullptr,
                            const ChemT<double>* b0 = nullptr, const CoolT<double>* k0 = nullptr) {
  const double yn[3] = {s.Tmu, s.xH2, s.xHp};
  const double Kinv = 1.0 / c.K;
  double y[3] = {yn[0], yn[1], yn[2]};
  int it = -1;
  Equil<double> qb;
  if (seed) {
    y[0] = seed[0]; y[1] = seed[1]; y[2] = seed[2];
    double xg = xe_g, tg = td_g;
    int spent = 0;
    it = cf ? chord64_from_seed<LPC>(c, *cf, p, s.mu, Kinv, yn, dts, y, xg, tg, &qb, &spent)
            : newton_solve<LPC>(c, p, s.mu, Kinv, yn, dts, y, xg, tg, (SEED_MAXIT < p.newton_max) ? SEED_MAXIT : p.newton_max,
                                &qb, &spent);
    if (it >= 0) {
      xe_g = xg; td_g = tg;
      s.status |= ST_SEEDED;
    } else {
      s.iters += spent;   // the abandoned seeded iterations count too
      s.status |= ST_SEED_FAIL;
    }
  }
  // b0, k0: the temperature blocks at the start state, if the caller has them
  if (it < 0) it = solve_from_start64<LPC>(c, p, s.mu, Kinv, yn, dts, y, xe_g, td_g, s.status, &qb, b0, k0);
  int halv = 0;
  while (it < 0 && halv < 30) {
    s.status |= ST_NEWTON;
    dts *= 0.5;
    last = false;
    ++halv;
    it = solve_from_start64<LPC>(c, p, s.mu, Kinv, yn, dts, y, xe_g, td_g, s.status, &qb, b0, k0);
  }
  if (it < 0) {
    s.status |= ST_NONFIN;
    s.t = dt;
    return;
  }
  s.iters += it;
  finish_substep_q(c, p, dt, dts, last, y, qb, s);
}

// Substep length of Sec. 6.1 from the source terms at the substep start, evaluated in
// precision F (FP64, or df64 in the mixed modes); K is the cell's FP64 heat-capacity
// factor.  `src`, when given, receives those terms (H, C_H2, C_H+).
template <class F>
TCG_FN double substep_start_t(const CellC<F>& cc, double K, const DevParams& p, double dt, const LaneState& s,
                              F& td_g, bool& last, double* src = nullptr, ChemT<F>* bo = nullptr,
                              CoolT<F>* ko = nullptr) {
  double H0, CH2, CHp;
  start_sources<F>(cc, p, s, td_g, H0, CH2, CHp, bo, ko);
  if (src) { src[0] = H0; src[1] = CH2; src[2] = CHp; }
  return substep_len(p, dt - s.t, K * s.Tmu, H0, CH2, CHp, last);
}
TCG_FN double substep_start64(const CellC<double>& c, const DevParams& p, double dt, const LaneState& s,
                              double& td_g, bool& last, double* src = nullptr, ChemT<double>* bo = nullptr,
                              CoolT<double>* ko = nullptr) {
  return substep_start_t<double>(c, c.K, p, dt, s, td_g, last, src, bo, ko);
}

template <int LPC = 1>
TCG_FN void substep_newton64(const CellC<double>& c, const DevParams& p, double dt, LaneState& s, double& xe_g,
                             double& td_g) {
  bool last;
  if constexpr (LPC == 1) {
    // the start's temperature blocks serve the first Newton iteration (same T)
    ChemT<double> b0;
    CoolT<double> k0;
    const double dts = substep_start64(c, p, dt, s, td_g, last, nullptr, &b0, &k0);
    solve_substep64<LPC>(c, p, dt, dts, last, s, xe_g, td_g, nullptr, nullptr, &b0, &k0);
  } else {
    const double dts = substep_start64(c, p, dt, s, td_g, last);
    solve_substep64<LPC>(c, p, dt, dts, last, s, xe_g, td_g);
  }
}

// ------------------------------------------------------------------ mode 2: mixed precision
// Mixed Newton on the same residual: FP32 source evaluations, FP64 residual, solve and
// update.  The forward-difference Jacobian (relative step 1e-3, large enough that FP32
// rounding in f stays ~1e-4 of each column) is built at the first iteration and reused;
// it is rebuilt (at most twice) when the steps contract by less than a factor 0.3.
// Returns the iteration count with polish = false when every step fell below
// rtol_mixed |y_i| (+1e-12 for the abundances); with polish = true when the steps
// stopped contracting above that, at the FP32 rounding floor of f (below 1e-4
// relative), which happens near stiff equilibria where H or C_s is a small difference
// of large terms; or -1 if neither happened.  J holds the last Jacobian on return.
template <int LPC = 1>
TCG_FN int newton_mixed(const CellC<float>& cf, const DevParams& p, double mu, double Kinv, const double* yn,
                        double dts, double* y, float& xe_g, float& td_g, float J[3][3], bool& polish,
                        int maxit = 0, int* spent = nullptr) {
  bool haveJ = false;
  int rebuilt = 0;
  float prev = 3e38f;
  polish = false;
  const int nmax = (maxit > 0 && maxit < p.newton_max) ? maxit : p.newton_max;
  for (int it = 1; it <= nmax; ++it) {
    if (spent) *spent = it;
    TCG_COUNT_D(newton32_it);
    double f0[3];
    bool coop = false;
    if (LPC == 4 && !haveJ) {
      // Warp-cooperative FP32 Jacobian: lane q evaluates f at the base point (q = 0) or
      // with x_H2, x_H+ or T_mu perturbed (q = 1, 2, 3); the results are exchanged.
      const int q = lane_in_cell<LPC>();
      const double h0 = 1e-3 * y[0];
      const double h1 = fmax(1e-3 * fabs(y[1]), 1e-12), h2 = fmax(1e-3 * fabs(y[2]), 1e-12);
      float xg = xe_g, tg = td_g;
      double fq[3];
      {
        ChemT<float> b = chem_T(cf, float(mu * ((q == 3) ? y[0] + h0 : y[0])), p.flags);
        CoolT<float> k = cool_T(cf, b, p.flags);
        feval32(cf, b, k, y[1] + ((q == 1) ? h1 : 0.0), y[2] + ((q == 2) ? h2 : 0.0), Kinv, xg, tg, fq);
      }
      const float s0 = float(dts) / float(h0), s1 = float(dts) / float(h1), s2 = float(dts) / float(h2);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        f0[i] = from_lane<LPC>(fq[i], 0);
        const double f1 = from_lane<LPC>(fq[i], 1), f2 = from_lane<LPC>(fq[i], 2), fT = from_lane<LPC>(fq[i], 3);
        J[i][1] = ((i == 1) ? 1.f : 0.f) - s1 * float(f1 - f0[i]);
        J[i][2] = ((i == 2) ? 1.f : 0.f) - s2 * float(f2 - f0[i]);
        J[i][0] = ((i == 0) ? 1.f : 0.f) - s0 * float(fT - f0[i]);
      }
      xe_g = from_lane<LPC>(xg, 0);
      td_g = from_lane<LPC>(tg, 0);
      haveJ = true;
      coop = true;
    }
    if (!coop) {
    ChemT<float> b = chem_T(cf, float(mu * y[0]), p.flags);
    CoolT<float> k = cool_T(cf, b, p.flags);
    feval32(cf, b, k, y[1], y[2], Kinv, xe_g, td_g, f0);
    if (!haveJ) {
#pragma unroll 1
      for (int j = 1; j < 3; ++j) {
        const double h = fmax(1e-3 * fabs(y[j]), 1e-12);
        const double y1 = y[1] + ((j == 1) ? h : 0.0), y2 = y[2] + ((j == 2) ? h : 0.0);
        float xg = xe_g, tg = td_g;
        double fx[3];
        feval32(cf, b, k, y1, y2, Kinv, xg, tg, fx);
        const float sj = float(dts) / float(h);
        for (int i = 0; i < 3; ++i) J[i][j] = ((i == j) ? 1.f : 0.f) - sj * float(fx[i] - f0[i]);
      }
      const double h = 1e-3 * y[0];
      ChemT<float> bT = chem_T(cf, float(mu * (y[0] + h)), p.flags);
      CoolT<float> kT = cool_T(cf, bT, p.flags);
      float xg = xe_g, tg = td_g;
      double fT[3];
      feval32(cf, bT, kT, y[1], y[2], Kinv, xg, tg, fT);
      const float s0 = float(dts) / float(h);
      for (int i = 0; i < 3; ++i) J[i][0] = ((i == 0) ? 1.f : 0.f) - s0 * float(fT[i] - f0[i]);
      haveJ = true;
    }
    }
    // residual in FP64 (a difference of nearby values), the correction solved in FP32
    float Jw[3][3], rhs[3], d32[3];
    for (int i = 0; i < 3; ++i) {
      rhs[i] = float(-(y[i] - yn[i] - dts * f0[i]));
      for (int j = 0; j < 3; ++j) Jw[i][j] = J[i][j];
    }
    if (!solve3_ool(Jw, rhs, d32)) return -1;
    const double d[3] = {double(d32[0]), double(d32[1]), double(d32[2])};
    double st[3];
    const bool full = damped_step_ool(y, d, st);
    // the convergence measure in FP32 (a ratio of step to tolerance)
    float nrm = 0.f;
    const float rtm = float(p.rtol_mixed);
    for (int i = 0; i < 3; ++i)
      nrm = fmaxf(nrm, fabsf(float(st[i])) / (rtm * fabsf(float(y[i])) + ((i == 0) ? 1e-30f : 1e-12f)));
    if (!finite3(y[0], y[1], y[2])) return -1;
    if (full) {
      if (nrm <= 1.f) return it;
      if (it >= 2 && nrm > 0.3f * prev) {
        if (nrm > 0.7f * prev && nrm * rtm <= 1e-4f) {
          polish = true;
          return it;
        }
        if (rebuilt < 2) {
          ++rebuilt;
          haveJ = false;
        }
      }
    }
    prev = nrm;
  }
  return -1;
}

// High-precision polish of the mixed iteration's root: chord corrections with the
// residual's source terms evaluated in df64 (double-float, ~1e-12 relative on the
// terms, tc_df64.cuh) and the last (FP32-built) Jacobian.  The FP32 root is off the FP64
// one by the FP32 rounding floor of f (~1e-6 relative in T near stiff equilibria, where
// H is a small difference of large terms), and the scheme can amplify such errors a
// hundredfold over a step, so every substep is polished.  With F = double the same
// polish runs in FP64; df64 gives the same roots to ~1e-11 relative (the terms' errors
// divided by the logarithmic slope of H in T) at a fraction of the FP64 pipe's time.
// The Jacobian is the FP32 forward difference built at the FP32 root (fd_jacobian32).
// A chord iteration contracts by the Jacobian's relative error rho (~1e-3 there), so
// after a correction d_k the remaining error is about rho d_k / (1 - rho), with rho
// estimated as d_k / d_(k-1).  Accepted when that estimate is below 1e-9 relative
// (abundances relative to max(x, 1e-4)), or when a single correction is below 3e-8;
// after at most five corrections, otherwise the FP64 solver takes the substep.
// Measured on 4 x 4096 random-state cells, largest error in T against the FP64 oracle
// after one step, and polish evaluations per slab substep:
//   Jacobian from the FP32 iteration, single correction below 1e-8: 4.6e-6, 1.83
//   (below 1e-7: 1.05e-5, 1.13, over the bound);
//   Jacobian rebuilt at the FP32 root, single correction below 1e-7: 1.1e-6, 1.15;
//   below 3e-8: 1.48 evaluations.  On a PDR slab run for 120 steps of 1 Myr the
//   largest error fell from 1.5e-6 (1e-7) to 1.1e-9 (3e-8; 1e-8 gave 1.2e-9): a
//   correction just under 1e-7 left an error that the cold molecular gas amplified
//   over the following steps.
// `qlast` receives the C/O/e equilibrium of the last evaluation.
template <class F>
TCG_FN bool polish_hp(const CellC<F>& c, const DevParams& p, double mu, double Kinv, const double* yn, double dts,
                      double* y, const float J[3][3], F& xe_g, F& td_g, Equil<F>& qlast) {
  double prev = -1.0;
  for (int it = 0; it < 5; ++it) {
    TCG_COUNT_D(polish_it);
    ChemT<F> b = chem_T(c, to_prec<F>(mu * y[0]), p.flags);
    CoolT<F> k = cool_T(c, b, p.flags);
    double f0[3];
    feval_t<F>(c, b, k, y[1], y[2], Kinv, xe_g, td_g, f0, &qlast);
    // FP64 residual; the correction (below ~1e-6 relative) solved in FP32 with the FP32
    // Jacobian, whose own error (~1e-3) sets the contraction
    float Jw[3][3], rhs[3], d32[3];
    for (int i = 0; i < 3; ++i) {
      rhs[i] = float(-(y[i] - yn[i] - dts * f0[i]));
      for (int j = 0; j < 3; ++j) Jw[i][j] = J[i][j];
    }
    if (!solve3_ool(Jw, rhs, d32)) return false;
    const double d[3] = {double(d32[0]), double(d32[1]), double(d32[2])};
    double st[3];
    const bool full = damped_step_ool(y, d, st);
    double nrm = 0.0;
    for (int i = 0; i < 3; ++i) nrm = fmax(nrm, fabs(st[i]) / (fabs(y[i]) + ((i == 0) ? 1e-300 : 1e-4)));
    if (!finite3(y[0], y[1], y[2])) return false;
    if (!full) {
      prev = -1.0;
      continue;
    }
    if (nrm <= 3e-8) return true;
    if (prev > 0.0) {
      const double rho = nrm / prev;
      if (rho < 0.5 && rho * nrm <= 1e-9 * (1.0 - rho)) return true;
    }
    prev = nrm;
  }
  return false;
}

// One mixed-precision substep.  High-precision work, in df64: the source terms at the
// substep start that set its length (Sec. 6.1; the length decides where the trajectory
// is sampled: FP32 heating and cooling sums are off by up to ~5e-5 relative, and a
// length that far off moved hot cells cooling through the Lyman-alpha peak by 1e-3 in T
// after ~70 substeps), and the polish of the root, whose last evaluation also gives the
// C/O/e equilibrium that sets mu at the end (finish_substep_q).  FP32 work: every Newton
// iteration before the polish and the Jacobian.  FP64 work: the Newton updates and
// residuals, and the fallback.  The solve starts from `seed` when given, else from the
// start state.
template <int LPC = 1>
TCG_FN void substep_mixed_solve(const CellC<double>& c, const CellC<df64>& cd, const CellC<float>& cf,
                                const DevParams& p, double dt, double dts, bool last, LaneState& s, float& xe_g,
                                float& td_g, const df64& td_hp, const double* seed) {
  const double yn[3] = {s.Tmu, s.xH2, s.xHp};
  const double Kinv = 1.0 / c.K;
  double y[3] = {yn[0], yn[1], yn[2]};
  if (seed) { y[0] = seed[0]; y[1] = seed[1]; y[2] = seed[2]; }
  float J[3][3];
  bool polish = false;
  int spent = 0;
  int it = newton_mixed<LPC>(cf, p, s.mu, Kinv, yn, dts, y, xe_g, td_g, J, polish, seed ? SEED_MAXIT : 0, &spent);
  if (seed) s.status |= (it >= 0) ? ST_SEEDED : ST_SEED_FAIL;
  if (it < 0 && seed) {
    // a seed that did not lead to convergence within SEED_MAXIT iterations: start again
    // from the start state (the abandoned iterations count too)
    s.iters += spent;
    y[0] = yn[0]; y[1] = yn[1]; y[2] = yn[2];
    it = newton_mixed<LPC>(cf, p, s.mu, Kinv, yn, dts, y, xe_g, td_g, J, polish);
  }
  Equil<df64> qlast;
  const int it32 = it;
  bool have32 = false;
  double y32[3];
  if (it >= 0) {
    if (polish) s.status |= ST_POLISH;
    y32[0] = y[0]; y32[1] = y[1]; y32[2] = y[2];
    have32 = true;
    fd_jacobian32<LPC>(cf, p, s.mu, Kinv, dts, y, xe_g, td_g, J);
    df64 xg = df64::make(xe_g, 0.0f), tg = df64::make(td_g, 0.0f);
    if (!polish_hp<df64>(cd, p, s.mu, Kinv, yn, dts, y, J, xg, tg, qlast)) it = -1;
  }
  if (it < 0) {
    // The plain FP64 solver finishes this substep (same length, same start state): when
    // the FP32 iteration converged and only its polish failed (an FP32 Jacobian too poor
    // near a singular one, in thermally unstable gas), first by Newton from that FP32
    // root, the root the polish was refining; otherwise, or if that fails, as mode 1
    // does (from the start state, the predictor, then half lengths).
    s.status |= ST_FALLBACK;
    double xg = s.xe, tg = double(td_hp);
    int it64 = -1;
    Equil<double> qb;
    if (have32) {
      y[0] = y32[0]; y[1] = y32[1]; y[2] = y32[2];
      it64 = newton_solve<LPC>(c, p, s.mu, Kinv, yn, dts, y, xg, tg, 0, &qb);
    }
    if (it64 >= 0) {
      s.iters += it32 + it64;
      finish_substep_q(c, p, dt, dts, last, y, qb, s);
    } else {
      xg = s.xe;
      tg = double(td_hp);
      solve_substep64<LPC>(c, p, dt, dts, last, s, xg, tg);
    }
  } else {
    s.iters += it;
    finish_substep_q(c, p, dt, dts, last, y, equil64(qlast), s);
  }
  xe_g = float(s.xe);
}

template <int LPC = 1>
TCG_FN void substep_mixed(const CellC<double>& c, const CellC<df64>& cd, const CellC<float>& cf, const DevParams& p,
                          double dt, LaneState& s, float& xe_g, float& td_g, df64& td_hp) {
  bool last;
  const double dts = substep_start_t<df64>(cd, c.K, p, dt, s, td_hp, last);
  substep_mixed_solve<LPC>(c, cd, cf, p, dt, dts, last, s, xe_g, td_g, td_hp, nullptr);
}

// ------------------------------------------------------------------ seeding (modes 3, 4)
// Features of a substep's seed: the substep start's state, the per-cell features
// lf[6] = log10 n, log10 chi_FUV, log10 f_shld,H2, log10(F_LyC+1), log10 xi, log10 Z'_d,
// the substep length, and the explicit-Euler changes over the substep from the
// start-state source terms src = (H, C_H2, C_H+) that set its length:
// g = dts (C_H2 / 0.5, C_H+, H / (K T_mu ln 10)).  Lanes without a substep (need false)
// get zeros: they take part in the warp's inference and ignore its output.
TCG_FN void seed_features(const float* lf, const CellC<double>& c, const LaneState& s, double dts, const double* src,
                          bool need, double* g, float* f) {
  if (!need) {
    for (int k = 0; k < MLP_IN; ++k) f[k] = 0.f;
    g[0] = g[1] = g[2] = 0.0;
    return;
  }
  g[0] = dts * src[1] / 0.5;
  g[1] = dts * src[2];
  g[2] = dts * src[0] / (c.K * s.Tmu) / LN10;
  const float v[MLP_IN] = {lf[0], (float)log10(s.mu * s.Tmu), (float)s.xH2, (float)s.xHp, lf[1], lf[2], lf[3], lf[4],
                           (float)log10(dts), lf[5], (float)g[0], (float)g[1], (float)g[2]};
  for (int k = 0; k < MLP_IN; ++k) f[k] = v[k];
}

// Seed from the network's outputs o (the backward-Euler changes beyond the explicit
// ones g): the prediction g + o mapped to (T_mu, x_H2, x_H+) with mu frozen at the
// substep start and clamped inside the admissible region.  Returns false (no seed) if
// it is not finite or leaves the trust region below.
TCG_FN bool seed_from_outputs(const float* o, const double* g, const LaneState& s, const DevParams& p,
                              double* seed) {
  const double d0 = g[0] + (double)o[0], d1 = g[1] + (double)o[1], d2 = g[2] + (double)o[2];
  if (!(isfinite(d0) && isfinite(d1) && isfinite(d2))) return false;
  // Trust region: the backward-Euler system can have several roots (thermally unstable
  // gas), and the solver's root is the one Newton reaches from the start state.  A seed
  // is used only when it predicts a small change, inside the basin of that root.
  if (fabs(d2) > SEED_MAX_DLOGT || fabs(0.5 * d0) > SEED_MAX_DX || fabs(d1) > SEED_MAX_DX) return false;
  const double T0 = s.mu * s.Tmu;
  const double x2 = fmin(fmax(s.xH2 + 0.5 * d0, 1e-20), 0.4999999);
  const double xp = fmin(fmax(s.xHp + d1, 1e-20), 0.999999 * (1.0 - 2.0 * x2));
  const double T1 = fmin(fmax(T0 * exp10(fmin(fmax(d2, -6.0), 6.0)), p.T_floor), 1e10);
  seed[0] = T1 / s.mu;
  seed[1] = x2;
  seed[2] = xp;
  return true;
}

// ------------------------------------------------------------------ the kernel
// Registers: 128 threads per block and at least 8 resident blocks per SM (64 registers
// per thread, the rest spilled to L1).  More resident warps hide more of the latency of
// these long dependent FP64 chains than the spills cost.  Measured on the 128^3 slab
// (FP64 Newton / mixed, ms):
//   3 blocks (168 registers, compiler's choice) 546 / 403
//   4 blocks (128) 394 / 195,  5 (96) 375 / 174,  6 (80) 365 / 164,
//   7 (72) 362 / 156,  8 (64) 363 / 152.
// With the FP64 exp and log out of line (a shorter per-thread stack) the autotuner picks
// 4 resident blocks of 128 for FP64 Newton and the paper scheme, and their kernels are
// compiled for 6 (80 registers): FP64 Newton 214.6 -> 212.9 ms, paper scheme 50.9 ->
// 50.0 (4 blocks: 214.1 / 50.7, 5: 213.3 / 50.3).  The seeded FP64 kernel keeps 8
// (293.5 ms; 300.1 at 6).
constexpr int STEP_MIN_BLOCKS = 8;
constexpr int STEP_MIN_BLOCKS_FP64 = 6;
// The warp-cooperative kernels (four lanes per cell) serve launches too small to fill
// the GPU, where the time is the latency of the slowest cells: 4 resident blocks (128
// registers per thread) spill less.
constexpr int STEP_MIN_BLOCKS_COOP = 4;

// The mixed kernels (modes 2, 3) are bound by latency rather than a pipe (instruction
// fetch, dependent df64 chains), and more resident warps hide more of it than the extra
// spills cost: 12 blocks per SM (40 registers per thread).  Measured on the 128^3 slab,
// mixed / seeded mixed ms: 8 blocks 67.1 / 56.6, 10: 58.6 / 52.6, 12: 58.1 / 51.0,
// 16: 57.9 / 52.7.
constexpr int STEP_MIN_BLOCKS_MIXED = 12;

template <int MODE, bool BATCH, int LPC = 1>
__global__ void __launch_bounds__(128, (LPC == 1) ? ((MODE == 2 || MODE == 3) ? STEP_MIN_BLOCKS_MIXED
                                                      : (MODE == 0 || MODE == 1) ? STEP_MIN_BLOCKS_FP64
                                                                              : STEP_MIN_BLOCKS)
                                                  : STEP_MIN_BLOCKS_COOP)
    k_step(DevFields f1, const BoxTable* __restrict__ boxes, DevParams p, double dt, unsigned long long* cursor,
           long long ntotal, const MlpDev* __restrict__ mlp) {
  static_assert(LPC == 1 || ((MODE == 1 || MODE == 2) && !BATCH), "cooperative kernels: modes 1 and 2, one box");
  constexpr bool SEEDED = (MODE == 3 || MODE == 4);
  constexpr bool MIXED = (MODE == 2 || MODE == 3);
  (void)mlp;  // the seeded modes read the network in its tensor-core layout, p.mlp_mma
  float lf[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  LaneState s;
  CellC<double> c;
  CellC<float> cf;   // FP32 copy of the cell constants (mixed and seeded modes)
  CellC<df64> cd;    // df64 copy (mixed modes: substep-start sources and polish)
  double xe_g = -1.0, td_g = -1.0;
  float xe_gf = -1.f, td_gf = -1.f;
  df64 td_hp = df64(-1.0);   // dust-temperature guess of the df64 evaluations
  DevFields fb;
  long long li = -1;   // local cell index within its box
  bool have = false;
  bool done = false;   // the work queue is empty for this lane
  while (true) {
    if (!have && !done) {
      long long gi = claim_cells_lpc<LPC>(cursor);
      if (gi >= ntotal) {
        done = true;
      } else {
        if (p.order) gi = (long long)p.order[gi];
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
        s.t = 0.0;
        s.xH2 = x20; s.xHp = xp0;
        s.Td = -1.0;
        s.nsub = 0;
        s.status = 0;
        s.iters = 0;
        if constexpr (MIXED) {
          // initial C/O/e equilibrium (it sets mu and hence T_mu): in df64 in the mixed
          // modes, whose FP64 physics then runs only in their rare fallbacks
          cd = cast_cell<df64>(c);
          ChemT<df64> b0 = chem_T(cd, to_df64(T0), p.flags);
          Equil<df64> q0 = equilibrium(cd, b0, to_df64(x20), to_df64(xp0), df64(-1.0));
          s.xe = double(q0.xe); s.xCp = double(q0.xCp); s.xCO = double(q0.xCO);
          xe_g = s.xe;
          td_g = -1.0;
        } else {
          // in FP64 in the FP64 modes
          ChemT<double> b0 = chem_T(c, T0, p.flags);
          Equil<double> q0 = equilibrium(c, b0, x20, xp0, -1.0);
          s.xe = q0.xe; s.xCp = q0.xCp; s.xCO = q0.xCO;
          xe_g = q0.xe;
          td_g = -1.0;
        }
        if constexpr (MIXED || SEEDED) {
          cf = cast_cell<float>(c);
          xe_gf = float(s.xe);
          td_gf = -1.f;
        }
        if constexpr (MIXED) td_hp = df64(-1.0);
        if constexpr (SEEDED) {
          const double chi_fuv = (1.8e-4 * fb.chi_pe[li] + 3.0e-5 * fb.chi_lw[li]) / 2.1e-4;
          const double Fl = fb.Flyc ? fb.Flyc[li] : 0.0;
          lf[0] = (float)log10(fb.n[li]);
          lf[1] = (float)log10(fmax(chi_fuv, 1e-30));
          lf[2] = (float)log10(fmax(fb.fh2[li], 1e-30));
          lf[3] = (float)log10(Fl + 1.0);
          lf[4] = (float)log10(fmax(fb.xi[li], 1e-30));
          lf[5] = (float)log10(fmax(fb.Zd ? fb.Zd[li] : fb.Zd_val, 1e-30));
        }
        s.mu = c.muH / (1.1 + s.xe - x20);
        s.Tmu = T0 / s.mu;
        have = true;
      }
    }
    if constexpr (SEEDED) {
      // The seed network runs on the warp's tensor cores, an instruction all 32 lanes
      // issue together: lanes stay in the loop until the whole warp is done.
      if (__all_sync(0xffffffffu, done)) break;
      bool need = false, last = false;
      double dts = 0.0, src[3] = {0.0, 0.0, 0.0}, g[3];
      if (have && s.t < dt) {
        if (s.nsub >= p.max_sub) {
          s.status |= ST_MAX_SUB;
          s.t = dt;
        } else {
          if constexpr (MODE == 3) dts = substep_start_t<df64>(cd, c.K, p, dt, s, td_hp, last, src);
          else dts = substep_start64(c, p, dt, s, td_g, last, src);
          need = true;
        }
      }
      float feat[MLP_IN], o[MLP_OUT];
      seed_features(lf, c, s, dts, src, need, g, feat);
      __syncwarp();
      mlp_infer_warp(p.mlp_mma, feat, o);
      if (need) {
        double seed[3];
        const bool ok = seed_from_outputs(o, g, s, p, seed);
        if constexpr (MODE == 3)
          substep_mixed_solve(c, cd, cf, p, dt, dts, last, s, xe_gf, td_gf, td_hp, ok ? seed : nullptr);
        else solve_substep64(c, p, dt, dts, last, s, xe_g, td_g, ok ? seed : nullptr, &cf);
        if (!finite3(s.Tmu, s.xH2, s.xHp)) {
          s.status |= ST_NONFIN;
          s.t = dt;
        }
      }
    } else {
      if (done) break;
      if (s.t < dt) {
        if (s.nsub >= p.max_sub) {
          s.status |= ST_MAX_SUB;
          s.t = dt;
        } else if constexpr (MODE == 0) {
          substep_paper(c, p, dt, s);
        } else if constexpr (MODE == 1) {
          substep_newton64<LPC>(c, p, dt, s, xe_g, td_g);
        } else if constexpr (MODE == 2) {
          substep_mixed<LPC>(c, cd, cf, p, dt, s, xe_gf, td_gf, td_hp);
        }
        if (!finite3(s.Tmu, s.xH2, s.xHp)) {
          s.status |= ST_NONFIN;
          s.t = dt;
        }
      }
    }
    if (have && !(s.t < dt)) {
      store_cell(fb, li, s);
      have = false;
    }
  }
}

}  // namespace tcg
