// Oracle for the per-cell thermochemistry source step of Kim, Gong, Kim & Ostriker
// (2023), "Photochemistry and Heating/Cooling of the Multiphase Interstellar Medium
// with UV Radiative Transfer for Magnetohydrodynamic Simulations" (arXiv:2210.08024).
//
// TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct FP64 CPU
// statement of what the step computes.  Only tests/, the smoke check and the CPU
// baseline leg of bench.py may call it; the library product path never does.  It
// shares no code, header, constant table or helper with the CUDA implementation.
//
// Every function is templated on the scalar type R so that the same source runs in
// plain double (R = double) and under an operation counter (R = oracle::Cnt from
// tc_opcount.hpp) that tallies the algorithmic FP64 work of the method.
//
// Citations name the paper's sections and equation labels.  Terms the paper cites
// but does not print ("closures") are defined in closures.md with their source;
// each is marked CLOSURE Cn below.  Readings of passages where the paper is silent
// are marked READING.
//
// Parity unpinned (labelled stand-ins that no printed number constrains beyond the
// equilibrium-curve shape): alpha_gr (C3), alpha_rrdr_C (C4), k_Cp_H2 (C5), x_MHp (C6),
// k_cd_H2_H/H2 (C7), k_H2s_H/H2 (C10), cool_rovib (C11), cool_CO (C17), the
// grain-recombination cooling (C18) and xe_He_cie / xe_metal_cie (C19).
#pragma once
#include <cmath>
#include <cstdint>

namespace oracle {

// ------------------------------------------------------------------ constants (cgs)
constexpr double kB = 1.380649e-16;      // erg/K
constexpr double eV = 1.602176634e-12;   // erg
constexpr double c_light = 2.99792458e10;
constexpr double a_rad = 7.57e-15;       // Sec. 4.3.6, radiation density constant as printed
constexpr double gamma_ad = 5.0 / 3.0;   // Sec. 2.2
constexpr double ln10 = 2.302585092994046;
constexpr double pc_cm = 3.0856775814913673e18;

// Flag bits (same meaning as the library's public flags, defined independently).
enum : unsigned {
  F_CONST_KGR = 1u,   // Sec. 7: tests use k_gr = 3e-17 Z'_d
  F_NO_ROVIB = 2u,    // Sec. 7.1.2: H2 ro-vibrational cooling off
  F_NO_CIE = 4u,      // CIE He+metal cooling term off
  F_FREEZE_T = 256u,  // oracle-only: hold T fixed (chemistry-only pins)
  F_PREDICTOR = 512u, // oracle-only: start every mode-B solve from the predictor (path pins)
};

// ST_PREDICTOR (informational): a substep's Newton solve was restarted from the predictor.
enum : int { ST_OK = 0, ST_MAX_SUBSTEPS = 1, ST_NEWTON = 2, ST_NONFINITE = 4, ST_PREDICTOR = 32 };

struct Params {
  double dvdr_kms_pc;          // <|dv/dr|> for CO LVG cooling, km/s/pc (Sec. 7.1.2 uses 1)
  double T_cmb;                // radiation temperature that floors dust heating (Sec. 4.3.6: 2.73 K)
  double chi0;                 // unattenuated FUV scale used for optical dust heating
  double opt_over_fuv;         // E_OPT,0 / E_FUV,0 (Sec. 4.3.6: ~1)
  double tau_opt_over_tau_pe;  // tau_OPT / tau_PE (Sec. 4.3.6: 1/3; Sec. 7.1.2: 1/1.87)
  double limiter;              // 0.1 in the substep rule (Sec. 6.1)
  double fd_rel_step;          // relative FD step for dH/dT_mu (Sec. 6.1 leaves it open)
  double newton_rtol;          // coupled-implicit (mode B) Newton tolerance
  double T_floor;              // lower bound on T after a temperature update
  int newton_max;
  int max_substeps;
  int mode;                    // 0 = the paper's sequential scheme, 1 = coupled implicit
  unsigned flags;
};

struct CellIn {  // one cell's frozen inputs (Table 1 parameters)
  double n;       // n_H [cm^-3]
  double chi_pe;  // chi_PE (Draine units)
  double chi_lw;  // chi_LW: dust-attenuated LW intensity (no self-shielding)
  double f_h2;    // f_shld,H2,eff ; chi_H2 = chi_LW f_shld,H2,eff (Eq. e:chi_H2)
  double f_c;     // f_shld,C,eff  ; chi_C = chi_LW f_shld,C,eff (Sec. 5.1)
  double F_lyc;   // ionising photon number flux c E_LyC / (h nu_LyC) [cm^-2 s^-1]
  double xi;      // primary CR ionisation rate per H [s^-1]
  double Zg, Zd;  // scaled gas metallicity and dust abundance
};

// ------------------------------------------------------------------ small helpers
template <class R> inline R rmax(R a, R b) { return (a < b) ? b : a; }
template <class R> inline R rmin(R a, R b) { return (b < a) ? b : a; }
template <class R> inline R rabs(R a) { return (a < R(0.0)) ? R(0.0) - a : a; }
template <class R> inline R log10_(R x) { using std::log; return log(x) / R(ln10); }
template <class R> inline R exp10_(R x) { using std::exp; return exp(x * R(ln10)); }
template <class R> inline R logistic(R z) { using std::exp; return R(1.0) / (R(1.0) + exp(R(0.0) - z)); }
template <class R> inline bool finite_(R v) { return std::isfinite(double(v)); }

// ------------------------------------------------------------------ per-cell constants
// Density and radiation are frozen over the subcycle (Sec. 6.1), so everything that
// depends only on them is evaluated once per cell.
template <class R> struct Pre {
  R n, lnn;        // n_H and ln n_H
  R G0;            // 1.7 chi_FUV (Sec. 4.2) with chi_FUV of Eq. e:chi_FUV
  R zpd;           // 5.7e-11 chi_LW f_shld,H2 (Eq. eq:H2_pd)
  R zpiH, zpiH2;   // sigma_pi F_LyC (Eqs. e:H_pi, eq:H2_pi)
  R zpiC_rad;      // 3.43e-10 chi_C (Sec. 3.2.1, text value)
  R zcrC;          // 3.85 xi_cr (Sec. 3.2.1)
  R lnCO;          // ln n_CO,crit (Eq. e:CO_fit), +inf if xi or Z'_d is zero
  R qH2;           // q_cr,H2(n) in erg (CLOSURE C9)
  R Gd;            // dust radiative heating per H (Sec. 4.3.6)
  R xCtot, xOtot;  // 1.6e-4 Z'_g, 3.2e-4 Z'_g (Sec. 3.2)
  R muH, K;        // mu_H (Table 1) and K = n mu_H k_B/(gamma-1) (Eq. e:ODE1)
  R Ntilde_per_x;  // n_H / |dv/dr| in cm^-2 (km/s)^-1: Ntilde = x_CO * this (Sec. 4.3.2)
};

template <class R> Pre<R> prepare(const CellIn& c, const Params& p) {
  using std::log; using std::exp; using std::pow;
  Pre<R> P;
  P.n = R(c.n);
  P.lnn = log(P.n);
  R chi_fuv = (R(1.8e-4) * R(c.chi_pe) + R(3.0e-5) * R(c.chi_lw)) / R(2.1e-4);
  P.G0 = R(1.7) * chi_fuv;
  P.zpd = R(5.7e-11) * R(c.chi_lw) * R(c.f_h2);
  P.zpiH = R(3.1e-18) * R(c.F_lyc);
  P.zpiH2 = R(4.6e-18) * R(c.F_lyc);
  P.zpiC_rad = R(3.43e-10) * R(c.chi_lw) * R(c.f_c);
  P.zcrC = R(3.85) * R(c.xi);
  if (c.xi > 0.0 && c.Zd > 0.0) {
    R xi16 = R(c.xi) / R(1e-16);
    R chi13 = pow(R(c.chi_lw), R(1.0) / R(3.0));  // chi_CO = chi_LW (Sec. 3.2.1)
    P.lnCO = chi13 * log(R(4e3) * R(c.Zd) / (xi16 * xi16)) + log(R(50.0) * xi16 / pow(R(c.Zd), R(1.4)));
  } else {
    P.lnCO = R(INFINITY);
  }
  // CLOSURE C9: q_cr,H2 piecewise linear in log10 n between 10 and 18 eV.
  R ln10n = P.lnn / R(ln10);
  R q;
  if (ln10n < R(2.0)) q = R(10.0);
  else if (ln10n < R(4.0)) q = R(10.0) + R(1.5) * (ln10n - R(2.0));
  else if (ln10n < R(7.0)) q = R(13.0) + R(4.0 / 3.0) * (ln10n - R(4.0));
  else if (ln10n < R(10.0)) q = R(17.0) + (ln10n - R(7.0)) / R(3.0);
  else q = R(18.0);
  P.qH2 = q * R(eV);
  // Gamma_d,UV = sum_k sigma_d,k c E_k over PE, LW, LyC (Sec. 4.3.6) with the band
  // absorption cross sections of Sec. 2.4 (0.9, 1.5, 1.9 x 1e-21 Z'_d) and c E = 4 pi J.
  R Zd = R(c.Zd);
  const R fourpi = R(4.0 * M_PI);
  R g = R(0.9e-21) * Zd * fourpi * R(1.8e-4) * R(c.chi_pe) + R(1.5e-21) * Zd * fourpi * R(3.0e-5) * R(c.chi_lw) +
        R(1.9e-21) * Zd * R(c.F_lyc) * R(19.4 * eV);
  // Gamma_d,OPT = sigma_d,OPT c E_OPT with E_OPT = E_OPT,0 exp(-tau_OPT), tau_OPT = r tau_PE,
  // tau_PE = -ln(chi_PE/chi0) clipped at 0, E_OPT,0 = (E_OPT,0/E_FUV,0) chi0 E_FUV^Draine.
  if (p.opt_over_fuv > 0.0 && p.chi0 > 0.0) {
    R ratio = rmin(R(c.chi_pe) / R(p.chi0), R(1.0));
    R att = (ratio > R(0.0)) ? exp(R(p.tau_opt_over_tau_pe) * log(ratio)) : R(0.0);
    g = g + R(0.3e-21) * Zd * R(p.opt_over_fuv) * fourpi * R(2.1e-4) * R(p.chi0) * att;
  }
  P.Gd = g;
  P.xCtot = R(1.6e-4) * R(c.Zg);
  P.xOtot = R(3.2e-4) * R(c.Zg);
  P.muH = R(1.40) - R(0.02) * (R(c.Zg) - R(1.0));
  P.K = P.n * P.muH * R(kB) / R(gamma_ad - 1.0);
  P.Ntilde_per_x = (p.dvdr_kms_pc > 0.0) ? P.n / R(p.dvdr_kms_pc / pc_cm) : R(INFINITY);
  return P;
}

// Sec. 4.2: grain charging parameter psi = G0 sqrt(T)/n_e, plus 50 K^1/2 cm^3 as the
// paper adds in practice.  READING: the same psi serves the PE efficiency, the
// grain-assisted recombination rates and their cooling; n_e is floored at 1e-30 so
// that psi stays finite in gas with no free electrons.
template <class R> inline R psi_charge(R G0, R T, R ne) {
  using std::sqrt;
  return G0 * sqrt(T) / rmax(ne, R(1e-30)) + R(50.0);
}

// ------------------------------------------------------------------ rate coefficients
// Eq. e:H2form (Hollenbach & McKee 1979 shape, normalised by the paper).
template <class R> inline R k_gr(R T, double Zd, unsigned flags) {
  using std::sqrt;
  if (flags & F_CONST_KGR) return R(3.0e-17) * R(Zd);
  R T2 = T / R(100.0);
  R s = sqrt(T2);
  return R(3.0e-17) * R(Zd) * (R(2.0) * s) / (R(1.0) + R(0.4) * s + R(0.2) * T2 + R(0.08) * T2 * T2);
}

// CLOSURE C1: case-B radiative recombination of H+ (Draine 2011 Eq. 14.6 form).
template <class R> inline R alpha_rr_H(R T) {
  using std::log; using std::pow;
  R T4 = T / R(1e4);
  return R(2.54e-13) * pow(T4, R(-0.8163) - R(0.0208) * log(T4));
}

// CLOSURE C2: collisional ionisation H + e (Cen 1992 fit).
template <class R> inline R k_ci_H(R T) {
  using std::sqrt; using std::exp;
  return R(5.85e-11) * sqrt(T) * exp(R(-157809.1) / T) / (R(1.0) + sqrt(T / R(1e5)));
}

// CLOSURE C3: grain-assisted recombination (Weingartner & Draine 2001c form),
// alpha = 1e-14 C0 / (1 + C1 psi^C2 (1 + C3 T^C4 psi^(-C5 - C6 ln T))) Z'_d.
constexpr double WD_H[7] = {12.25, 8.074e-6, 1.378, 5.087e2, 1.586e-2, 0.4723, 1.102e-5};
constexpr double WD_C[7] = {45.58, 6.089e-3, 1.128, 4.331e2, 4.845e-2, 0.8120, 1.333e-4};
template <class R> inline R alpha_gr(R T, R lnT, R psi, double Zd, const double* C) {
  using std::pow;
  R inner = R(1.0) + R(C[3]) * pow(T, R(C[4])) * pow(psi, R(0.0) - R(C[5]) - R(C[6]) * lnT);
  return R(1e-14) * R(C[0]) / (R(1.0) + R(C[1]) * pow(psi, R(C[2])) * inner) * R(Zd);
}

// CLOSURE C4: C+ radiative + dielectronic recombination (stand-in power law).
template <class R> inline R alpha_rrdr_C(R T) { using std::pow; return R(4.67e-12) * pow(T / R(300.0), R(-0.6)); }
// CLOSURE C5: C+ + H2 -> CH2+ (stand-in radiative-association power law).
template <class R> inline R k_Cp_H2(R T) { using std::pow; return R(4.0e-16) * pow(T / R(300.0), R(-0.2)); }
// CLOSURE C7: collisional dissociation of H2 by H and by H2 (stand-ins).
template <class R> inline R k_cd_H2_H(R T) {
  using std::sqrt; using std::exp;
  return R(6.67e-12) * sqrt(T) * exp(R(0.0) - (R(1.0) + R(63593.0) / T));
}
template <class R> inline R k_cd_H2_H2(R T) {
  using std::pow; using std::exp;
  return R(5.996e-30) * pow(T, R(4.1881)) * exp(R(-54657.4) / T) / pow(R(1.0) + R(6.761e-6) * T, R(5.6881));
}
// CLOSURE C10: collisional de-excitation of H2* by H and by H2 (stand-ins).
template <class R> inline R k_H2s_H(R T) { using std::sqrt; using std::exp; return R(1.0e-12) * sqrt(T) * exp(R(-1000.0) / T); }
template <class R> inline R k_H2s_H2(R T) {
  using std::sqrt; using std::exp;
  return R(1.4e-12) * sqrt(T) * exp(R(-18100.0) / (T + R(1200.0)));
}
// CLOSURE C6: molecular-ion electrons (stand-in for Draine 2011 Eq. 16.25), times 2 x_H2
// as the paper prescribes (Sec. 3.3).
template <class R> inline R x_MHp(double xi, R n, R T, R xH2) {
  using std::sqrt; using std::pow;
  if (!(xi > 0.0)) return R(0.0);
  R aMH = R(2.4e-7) * pow(T / R(300.0), R(-0.69));
  return R(2.0) * xH2 * sqrt(R(1.67) * R(xi) / (aMH * n));
}

// ------------------------------------------------------------------ hot-gas stand-ins (CLOSURE C19)
template <class R> inline R gauss_bump(R lt, double mu, double sig) {
  using std::exp;
  R z = (lt - R(mu)) / R(sig);
  return exp(R(-0.5) * z * z);
}
template <class R> inline R xe_He_cie(R lt) {
  return R(0.1) * (logistic((lt - R(4.45)) / R(0.06)) + logistic((lt - R(4.95)) / R(0.06)));
}
template <class R> inline R xe_metal_cie(R lt) { return R(0.012) * logistic((lt - R(5.5)) / R(0.25)); }
template <class R> inline R Lambda_CIE(R lt, double Zg) {  // Eq. e:Lambda_CIE
  R LHe = R(2.0e-23) * gauss_bump(lt, 5.0, 0.15);
  R Lm = R(5.4e-22) * gauss_bump(lt, 5.35, 0.28) + R(5.0e-23) * gauss_bump(lt, 6.3, 0.35);
  return LHe + R(Zg) * Lm;
}

// Sec. 4.3: S(T) = 1/[1 + exp(-a (T - (T_t1+T_t2)/2)/(T_t2 - T_t1))], a = 10,
// T_t1 = 2e4 K, T_t2 = 3.5e4 K.
template <class R> inline R sigmoid_S(R T) {
  using std::exp;
  return R(1.0) / (R(1.0) + exp(R(-10.0) * (T - R(0.5) * (R(2e4) + R(3.5e4))) / (R(3.5e4) - R(2e4))));
}

// ------------------------------------------------------------------ equilibrium C/O/e (Secs. 3.2, 3.3)
template <class R> struct Equil {
  R xe, xCp, xCO, xC, xO, xOp, xMHp;
};

// Temperature-dependent, electron-independent pieces of the C+ balance.
template <class R> struct CpT {
  R src;   // zeta_pi,C + zeta_cr,C
  R arr;   // alpha_rr+dr,C+
  R sink0; // k_C+-H2 n_H2 (electron-independent sink, per s)
  R sqT, lnT, T;
};

// Eq. eq:C+_frac at a trial electron abundance xe.
template <class R> inline R xCp_of_xe(const Pre<R>& P, double Zd, const CpT<R>& k, R xe) {
  R ne = xe * P.n;
  R psi = P.G0 * k.sqT / rmax(ne, R(1e-30)) + R(50.0);
  R agr = alpha_gr(k.T, k.lnT, psi, Zd, WD_C);
  R den = k.src + agr * P.n + k.arr * ne + k.sink0;
  if (!(den > R(0.0))) return R(0.0);
  return P.xCtot * k.src / den;
}

// Electron abundance: Eq. e:xEL below 2e4 K and Eq. e:xELhot above, READING: blended
// with the cooling sigmoid S(T) since the paper only says "T >~ 2e4 K".  x_C+ depends on
// n_e through alpha_rr+dr,C+ n_e and alpha_gr,C+(psi(n_e)); g(x_e) = x_e - rhs(x_e) is
// strictly increasing, so the root on [a0, a0 + (1-S) x_C,tot] is unique.  Solved by
// the Illinois variant of regula falsi to a relative bracket width of 1e-14.
// Then CO (Eqs. e:CO, e:CO_fit), C and O by conservation, O+ = x_O,tot x_H+ (Sec. 3.2.2).
template <class R> inline Equil<R> equilibrium(const CellIn& c, const Pre<R>& P, R T, R xH2, R xHp) {
  using std::exp; using std::log; using std::sqrt;
  Equil<R> q;
  R lnT = log(T);
  R lt = lnT / R(ln10);
  R S = sigmoid_S(T);
  R w = R(1.0) - S;
  q.xOp = P.xOtot * xHp;
  q.xMHp = x_MHp(c.xi, P.n, T, xH2);
  R a_low = xHp + q.xOp + q.xMHp;
  R a_hot = xHp + xe_He_cie(lt) + R(c.Zg) * xe_metal_cie(lt);
  R a0 = w * a_low + S * a_hot;
  CpT<R> k;
  k.T = T; k.lnT = lnT; k.sqT = sqrt(T);
  // Sec. 3.2.1: zeta_pi,C = 3.43e-10 chi_C + 520 * 2 x_H2 xi_cr
  k.src = P.zpiC_rad + R(520.0) * R(2.0) * xH2 * R(c.xi) + P.zcrC;
  k.arr = alpha_rrdr_C(T);
  k.sink0 = k_Cp_H2(T) * P.n * xH2;
  R lo = a0, hi = a0 + w * P.xCtot;
  R xe;
  if (!(hi > lo)) {
    xe = a0;
  } else {
    R flo = lo - a0 - w * xCp_of_xe(P, c.Zd, k, lo);
    R fhi = hi - a0 - w * xCp_of_xe(P, c.Zd, k, hi);
    if (!(flo < R(0.0))) {
      xe = lo;
    } else if (!(fhi > R(0.0))) {
      xe = hi;
    } else {
      int side = 0;
      xe = lo;
      for (int it = 0; it < 200; ++it) {
        R x = (lo * fhi - hi * flo) / (fhi - flo);
        R fx = x - a0 - w * xCp_of_xe(P, c.Zd, k, x);
        xe = x;
        if (fx == R(0.0)) break;
        if (fx > R(0.0)) {
          hi = x; fhi = fx;
          if (side == 1) flo = flo * R(0.5);
          side = 1;
        } else {
          lo = x; flo = fx;
          if (side == -1) fhi = fhi * R(0.5);
          side = -1;
        }
        if (hi - lo <= R(1e-14) * hi) break;
      }
    }
  }
  q.xe = xe;
  q.xCp = xCp_of_xe(P, c.Zd, k, xe);
  R frac_ion = rmax((P.xCtot > R(0.0)) ? q.xCp / P.xCtot : R(0.0), xHp);
  R r2 = exp(R(2.0) * (P.lnCO - P.lnn));
  q.xCO = P.xCtot * R(2.0) * xH2 * (R(1.0) - frac_ion) / (R(1.0) + r2);
  q.xC = P.xCtot - q.xCp - q.xCO;
  q.xO = P.xOtot - q.xCO - q.xOp;
  return q;
}

// ------------------------------------------------------------------ hydrogen rates (Sec. 3.1)
template <class R> struct HRates {
  R kgr, zcrH2, zcrH, zcd, zci, arr, agr, kcdH, kcdH2, kci;
};

// Rate coefficients at (T, x_H2, x_H+, x_e); psi is psi_charge(G0, T, x_e n).
template <class R> inline HRates<R> h_rates(const CellIn& c, const Params& p, const Pre<R>& P, R T, R lnT, R xH2,
                                            R xHp, R xe, R psi) {
  HRates<R> r;
  R xH = R(1.0) - R(2.0) * xH2 - xHp;  // Sec. 3.1.3 (not clipped: f stays smooth; READING)
  r.kgr = k_gr(T, c.Zd, p.flags);
  r.zcrH2 = R(2.0) * R(c.xi) * (R(2.3) * xH2 + R(1.5) * xH);  // Eq. eq:H2_cr
  r.zcrH = r.zcrH2 / R(2.0);                                 // Sec. 3.1.2
  r.kcdH = k_cd_H2_H(T);
  r.kcdH2 = k_cd_H2_H2(T);
  r.zcd = r.kcdH * P.n * xH + r.kcdH2 * P.n * xH2;           // Sec. 3.1.1
  r.kci = k_ci_H(T);
  r.zci = r.kci * xe * P.n;                                  // Sec. 3.1.2
  r.arr = alpha_rr_H(T);
  r.agr = alpha_gr(T, lnT, psi, c.Zd, WD_H);
  return r;
}

// Eq. e:HH and Eq. e:HII.
template <class R> inline void h_sources(const HRates<R>& r, const Pre<R>& P, R xH2, R xHp, R xe, R& CH2, R& CHp) {
  R xH = R(1.0) - R(2.0) * xH2 - xHp;
  CH2 = r.kgr * P.n * xH - (R(1.65) * r.zcrH2 + P.zpd + P.zpiH2 + r.zcd) * xH2;
  CHp = (P.zpiH + r.zcrH + r.zci) * xH - (r.arr * xe * P.n + r.agr * P.n) * xHp;
}

// ------------------------------------------------------------------ dust temperature (Eq. eq:dust_en)
// Solves sigma_IR(T_d) c a (T_d^4 - T_cmb^4) = Gamma_d,UV + Gamma_d,OPT + n Lambda_g-d(T, T_d)
// with sigma_IR = 2e-25 Z'_d (T_d/10)^2: safeguarded Newton on a bracket
// [min(T, T_cmb), T_hi] where the residual changes sign.  READING: the CMB term is the
// paper's Gamma_d,CMB = sigma_IR c a T_CMB^4 moved to the left-hand side.
template <class R> inline R dust_temperature(const CellIn& c, const Params& p, const Pre<R>& P, R T, R sqT) {
  using std::pow;
  if (!(c.Zd > 0.0)) return T;
  R B = R(2e-27) * R(c.Zd) * R(c_light) * R(a_rad);  // sigma_IR c a = B T_d^2
  R Cc = P.n * R(3.2e-34) * R(c.Zd) * sqT;            // n alpha_g-d sqrt(T) Z'_d
  R Tc = R(p.T_cmb);
  R Tc4 = Tc * Tc * Tc * Tc;
  R lo = rmin(T, Tc);
  R hi = rmax(rmax(T, R(1.2) * Tc), pow(R(2.0) * P.Gd / B, R(1.0) / R(6.0)));
  R y = R(0.5) * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    R y2 = y * y;
    R h = B * y2 * (y2 * y2 - Tc4) - P.Gd - Cc * (T - y);
    if (h > R(0.0)) hi = y; else lo = y;
    R dh = B * (R(6.0) * y2 * y2 * y - R(2.0) * y * Tc4) + Cc;
    R yn = y - h / dh;
    if (!(yn > lo && yn < hi)) yn = R(0.5) * (lo + hi);
    R dy = rabs(yn - y);
    y = yn;
    if (dy <= R(1e-14) * y || hi - lo <= R(1e-14) * hi) break;
  }
  return y;
}

// ------------------------------------------------------------------ heating (Sec. 4.1)
template <class R> struct Heat {
  R pe, cr, pi, h2form, h2pump, h2pd, total;
};

// CLOSURE C8: energy per primary CR ionisation in atomic gas, 7.5..32 eV.
template <class R> inline R q_cr_H(R xe) {
  using std::sqrt;
  return (R(7.5) + R(24.5) * sqrt(xe / (xe + R(0.07)))) * R(eV);
}

template <class R> inline Heat<R> heating(const CellIn& c, const Pre<R>& P, const HRates<R>& r, R T, R xH2, R xHp,
                                          R xe, R psi) {
  using std::pow;
  Heat<R> h;
  R xH = R(1.0) - R(2.0) * xH2 - xHp;
  // Eq. eq:photoel_heat with Eq. e:PE_efficiency (C0..C6 as printed)
  R eps = (R(5.22) + R(2.25) * pow(T, R(0.147))) /
          (R(1.0) + R(0.04996) * pow(psi, R(0.431)) * (R(1.0) + R(0.00430) * pow(psi, R(0.692))));
  h.pe = R(1e-26) * P.G0 * eps * R(c.Zd);
  // Eq. eq:CR_heat with q_cr = x_H q_cr,H + 2 x_H2 q_cr,H2 (Sec. 4.3)
  h.cr = R(c.xi) * (xH * q_cr_H(xe) + R(2.0) * xH2 * P.qH2);
  // Eqs. eq:photoion_heat, eq:photoion_heat_H2 with q_pi,H = 3.4 eV, q_pi,H2 = 4.4 eV
  h.pi = xH * R(3.4 * eV) * P.zpiH + xH2 * R(4.4 * eV) * P.zpiH2;
  // Eqs. e:Gamma_H2form/pump/diss.  The factor 1/(1 + n_crit/n) with n_crit from Sec. 4.4
  // (A_eff = 2e-7 s^-1) is written as n d/(n d + A_eff + zeta_pd), d = x_H k_H + x_H2 k_H2.
  R dcoll = xH * k_H2s_H(T) + xH2 * k_H2s_H2(T);
  R fcoll = (P.n * dcoll) / (P.n * dcoll + R(2e-7) + P.zpd);
  h.h2form = r.kgr * P.n * xH * (R(0.2 * eV) + R(4.2 * eV) * fcoll);
  h.h2pump = P.zpd * xH2 * R(8.0) * R(2.0 * eV) * fcoll;
  h.h2pd = P.zpd * xH2 * R(0.4 * eV);
  h.total = h.pe + h.cr + h.pi + h.h2form + h.h2pump + h.h2pd;  // Eq. e:heating
  return h;
}

// ------------------------------------------------------------------ cooling (Sec. 4.3)
template <class R> struct Cool {
  R lya, ci, cd, rovib, ff, rr, hyd;
  R Cp, C, O, CO, grrec, neb, gd, cie, S, total;
};

// CLOSURE C14: two-level C+ 158 um.  Collision rates from the printed critical
// densities (Sec. 4.3.2): k_ul = A_ul/n_crit for e and H; H2 at half the H rate.
template <class R> inline R cool_Cp(R T, R lnT, R n, R xH, R xH2, R xe, R xCp) {
  using std::sqrt; using std::pow; using std::exp;
  const R A10 = R(2.3e-6), E10 = R(91.25);
  R T4 = T / R(1e4);
  R lnT2 = lnT - R(std::log(100.0));
  R ke = A10 / (R(53.0) * sqrt(T4));
  R kH = A10 / (R(3e3) * exp((R(-0.1281) - R(0.0087) * lnT2) * lnT2));
  R C10 = ke * xe * n + kH * xH * n + R(0.5) * kH * xH2 * n;
  R C01 = C10 * R(2.0) * exp(R(0.0) - E10 / T);
  R f1 = C01 / (A10 + C10 + C01);
  return xCp * f1 * A10 * E10 * R(kB) / n;
}

// CLOSURES C15, C16: three-level fine-structure atom.  k_10 from the printed n_crit
// anchors at 10 K and 5000 K (Sec. 4.3.2), power law in T between them;
// k_20 = k_21 = k_10; H2 collisions at half the H rate; electron collisions neglected.
template <class R> inline R cool_3level(R T, R lnT, R n, R xH, R xH2, R xs, double E1, double E2, double g0,
                                        double g1, double g2, double A10, double A20, double A21, double ncrit10,
                                        double ncrit5000) {
  using std::exp;
  const double s = std::log(ncrit5000 / ncrit10) / std::log(500.0);
  R ncrit = R(ncrit10) * exp(R(s) * (lnT - R(std::log(10.0))));
  R k10 = R(A10) / ncrit;
  R coll = (xH + R(0.5) * xH2) * n;
  R C10 = k10 * coll, C20 = k10 * coll, C21 = k10 * coll;
  R C01 = C10 * R(g1 / g0) * exp(R(0.0) - R(E1) / T);
  R C02 = C20 * R(g2 / g0) * exp(R(0.0) - R(E2) / T);
  R C12 = C21 * R(g2 / g1) * exp(R(0.0) - R(E2 - E1) / T);
  // statistical equilibrium of levels 1 and 2 relative to the ground level 0
  R a11 = R(A10) + C10 + C12;
  R b = R(A21) + C21;
  R a22 = R(A20) + R(A21) + C20 + C21;
  R det = a11 * a22 - b * C12;
  R r1 = (C01 * a22 + b * C02) / det;
  R r2 = (a11 * C02 + C12 * C01) / det;
  R z = R(1.0) + r1 + r2;
  R f1 = r1 / z, f2 = r2 / z;
  return xs * (f1 * R(A10) * R(E1) + f2 * (R(A20) * R(E2) + R(A21) * R(E2 - E1))) * R(kB) / n;
}

// CLOSURE C11: H2 ro-vibrational cooling: low-density limit (Galli & Palla 1998 fit)
// and LTE limit (Hollenbach & McKee 1979) combined harmonically; T clamped to [10, 1e4] K.
template <class R> inline R cool_rovib(R T, R n, R xH2) {
  using std::exp; using std::pow;
  R Tc = rmin(rmax(T, R(10.0)), R(1e4));
  R lt = log10_(Tc);
  R llow = R(-103.0) + lt * (R(97.59) + lt * (R(-48.05) + lt * (R(10.80) + lt * R(-0.9032))));
  R Llow = exp10_(llow);  // erg cm^3 s^-1 per H2 per H
  R T3 = Tc / R(1e3);
  R q = R(0.13) / T3;
  R Lrot = R(9.5e-22) * pow(T3, R(3.76)) / (R(1.0) + R(0.12) * pow(T3, R(2.1))) * exp(R(0.0) - q * q * q) +
           R(3e-24) * exp(R(-0.51) / T3);
  R Lvib = R(6.7e-19) * exp(R(-5.86) / T3) + R(1.6e-18) * exp(R(-11.7) / T3);
  R LLTE = Lrot + Lvib;
  R nL = n * Llow;
  R den = nL + LLTE;
  R L = (den > R(0.0)) ? (LLTE * nL / den) : R(0.0);
  return xH2 * L / n;
}

// CLOSURE C17: CO rotational cooling stand-in with LVG-like trapping through
// Ntilde = n_CO/|dv/dr| in cm^-2 (km/s)^-1 (Sec. 4.3.2 names the variable).
template <class R> inline R cool_CO(const Pre<R>& P, R T, R xCO) {
  using std::pow;
  R Nt = xCO * P.Ntilde_per_x;
  R t10 = T / R(10.0);
  R L = R(4e-27) * P.n * pow(t10, R(1.5)) / (R(1.0) + P.n / (R(3e3) * pow(t10, R(0.5))) + Nt / R(1e17));
  return xCO * L / P.n;
}

// Full cooling function, Eq. eq:cooling_fnct, at dust temperature Td.
template <class R> inline Cool<R> cooling(const CellIn& c, const Params& p, const Pre<R>& P, const HRates<R>& r, R T,
                                          R lnT, R sqT, R xH2, R xHp, const Equil<R>& q, R Td, R psi) {
  using std::pow; using std::exp;
  Cool<R> L;
  R n = P.n;
  R xe = q.xe;
  R xH = R(1.0) - R(2.0) * xH2 - xHp;
  R T4 = T / R(1e4);
  R lT4 = lnT - R(std::log(1e4));
  R lt = lnT / R(ln10);
  // Eq. e:k_lya; Lyman-alpha cooling x_H x_e E_21 k_12 with E_21/k_B = 1.184e5 K
  R k12 = R(5.31e-8) * exp(R(0.15) * lT4) / (R(1.0) + pow(T4 / R(5.0), R(0.65))) * exp(R(-11.84) / T4);
  L.lya = xH * xe * R(1.184e5 * kB) * k12;
  L.ci = R(13.6 * eV) * xH * xe * r.kci;                       // Eq. e:Lambda_ci_H
  L.cd = R(4.48 * eV) * xH2 * (xH * r.kcdH + xH2 * r.kcdH2);  // Eq. e:Lambda_cd_H2
  L.rovib = (p.flags & F_NO_ROVIB) ? R(0.0) : cool_rovib(T, n, xH2);
  R d = R(5.5) - lt;
  R gff = R(1.1) + R(0.34) * exp(R(0.0) - d * d / R(3.0));    // CLOSURE C12
  L.ff = R(1.42e-27) * sqT * gff * xe * xHp;
  L.rr = r.arr * R(kB) * T * (R(0.684) - R(0.0416) * lT4) * xe * xHp;  // CLOSURE C13
  L.hyd = L.lya + L.ci + L.rovib + L.cd + L.ff + L.rr;
  L.Cp = cool_Cp(T, lnT, n, xH, xH2, xe, q.xCp);
  // O: 3P2 ground (g 5), 3P1 at 227.7 K (g 3), 3P0 at 326.6 K (g 1).
  L.O = cool_3level(T, lnT, n, xH, xH2, q.xO, 227.7, 326.6, 5.0, 3.0, 1.0, 8.91e-5, 1.34e-10, 1.75e-5, 2.5e5, 4.9e4);
  // C: 3P0 ground (g 1), 3P1 at 23.6 K (g 3), 3P2 at 62.4 K (g 5).
  L.C = cool_3level(T, lnT, n, xH, xH2, q.xC, 23.6, 62.4, 1.0, 3.0, 5.0, 7.93e-8, 2.0e-14, 2.65e-7, 620.0, 150.0);
  L.CO = cool_CO(P, T, q.xCO);
  // CLOSURE C18: grain-assisted recombination cooling (Bakes & Tielens 1994 form).
  L.grrec = R(4.65e-30) * pow(T, R(0.94)) * pow(psi, R(0.74) / pow(T, R(0.068))) * xe * R(c.Zd);
  // Eq. e:Lambda_neb with log10 f_neb = sum a_i (ln T4)^i
  R ne2 = xe * n / R(100.0);
  R poly = R(6.92e-1) + lT4 * (R(-5.86e-1) + lT4 * (R(8.16e-1) + lT4 * (R(-5.05e-1) +
           lT4 * (R(1.18e-1) + lT4 * (R(7.66e-3) + lT4 * R(-5.08e-3))))));
  R fneb = exp10_(poly);
  R nden = exp(R(0.5) * lT4) * (R(1.0) + R(0.12) * pow(ne2, R(0.38) - R(0.12) * lT4));
  L.neb = R(c.Zg) * xe * xHp * R(3.68e-23) * exp(R(-3.86) / T4) * fneb / nden;
  L.gd = R(3.2e-34) * sqT * (T - Td) * R(c.Zd);  // Eq. eq:gas-dust
  L.S = sigmoid_S(T);
  L.cie = (p.flags & F_NO_CIE) ? R(0.0) : Lambda_CIE(lt, c.Zg);
  L.total = L.hyd + (R(1.0) - L.S) * (L.Cp + L.C + L.O + L.CO + L.grrec + L.neb + L.gd) + L.S * L.cie;
  return L;
}

// ------------------------------------------------------------------ net source terms
template <class R> struct Source {
  R H;  // net heating per volume n Gamma - n^2 Lambda [erg cm^-3 s^-1] (Eq. e:ODE1)
  R CH2, CHp;
  R Td;
  HRates<R> r;
  Heat<R> heat;
  Cool<R> cool;
};

// Evaluates H, C_H2, C_H+ at temperature T with abundances (x_H2, x_H+) and the
// equilibrium bundle q.  If Td_in > 0 it is used as the (frozen) dust temperature,
// otherwise the dust temperature is solved at T.
template <class R> inline Source<R> source_terms(const CellIn& c, const Params& p, const Pre<R>& P, R T, R xH2, R xHp,
                                                 const Equil<R>& q, R Td_in) {
  using std::log; using std::sqrt;
  Source<R> s;
  R lnT = log(T);
  R sqT = sqrt(T);
  R psi = P.G0 * sqT / rmax(q.xe * P.n, R(1e-30)) + R(50.0);
  s.r = h_rates(c, p, P, T, lnT, xH2, xHp, q.xe, psi);
  h_sources(s.r, P, xH2, xHp, q.xe, s.CH2, s.CHp);
  s.heat = heating(c, P, s.r, T, xH2, xHp, q.xe, psi);
  s.Td = (Td_in > R(0.0)) ? Td_in : dust_temperature(c, p, P, T, sqT);
  s.cool = cooling(c, p, P, s.r, T, lnT, sqT, xH2, xHp, q, s.Td, psi);
  s.H = P.n * s.heat.total - P.n * P.n * s.cool.total;
  return s;
}

template <class R> inline R mu_of(const Pre<R>& P, R xe, R xH2) { return P.muH / (R(1.1) + xe - xH2); }  // Sec. 2.2

// ------------------------------------------------------------------ results
struct CellOut {
  double T, xH2, xHp, xe, xCp, xCO;
  int nsub, status, newton_iters;
};

// Substep length rule of Sec. 6.1 truncated to the remaining time (READING).
template <class R> inline R substep_length(const Params& p, R rem, R e, R H, R CH2, R CHp, bool& last) {
  R dts = rem;
  R lim = R(p.limiter);
  R aH = rabs(H), a1 = rabs(CH2), a2 = rabs(CHp);
  if (aH > R(0.0)) dts = rmin(dts, lim * e / aH);
  if (a1 > R(0.0)) dts = rmin(dts, lim / a1);
  if (a2 > R(0.0)) dts = rmin(dts, lim / a2);
  last = !(dts < rem);
  if (last) dts = rem;
  return dts;
}

// ------------------------------------------------------------------ mode A: the paper's scheme (Sec. 6.1)
template <class R> CellOut step_paper(const CellIn& c, const Params& p, double T_in, double xH2_in, double xHp_in,
                                      double dt) {
  using std::log; using std::sqrt;
  CellOut out{};
  const Pre<R> P = prepare<R>(c, p);
  R xH2 = R(xH2_in), xHp = R(xHp_in);
  // READING: the initial x_e (and hence mu) is the equilibrium at the input temperature.
  Equil<R> q = equilibrium(c, P, R(T_in), xH2, xHp);
  R mu = mu_of(P, q.xe, xH2);
  R Tmu = R(T_in) / mu;
  R t = R(0.0);
  int nsub = 0, status = ST_OK;
  const R dtR = R(dt);
  bool done = !(dt > 0.0);
  while (!done) {
    if (nsub >= p.max_substeps) { status |= ST_MAX_SUBSTEPS; break; }
    R T = mu * Tmu;
    R e = P.K * Tmu;
    Source<R> s = source_terms(c, p, P, T, xH2, xHp, q, R(-1.0));
    bool last;
    R dts = substep_length(p, dtR - t, e, (p.flags & F_FREEZE_T) ? R(0.0) : s.H, s.CH2, s.CHp, last);
    // Temperature: linearised backward Euler with x (and mu, x_e, T_d) frozen and
    // dH/dT_mu by a forward difference of relative step fd_rel_step (READING).
    R Tmu_new = Tmu;
    if (!(p.flags & F_FREEZE_T) && s.H != R(0.0)) {
      R dTmu = R(p.fd_rel_step) * Tmu;
      Source<R> sp = source_terms(c, p, P, mu * (Tmu + dTmu), xH2, xHp, q, s.Td);
      R D = (sp.H - s.H) / dTmu;
      R tcool = R(0.0) - e / s.H;
      R r = dts / tcool;
      R den = R(1.0) + r * (Tmu / s.H) * D;
      if (den < R(0.1)) den = R(1.0);  // READING: explicit form when the denominator is small
      Tmu_new = Tmu * (R(1.0) + (R(0.0) - r) / den);
      R Tmu_floor = R(p.T_floor) / mu;  // READING: temperature floor
      if (Tmu_new < Tmu_floor) Tmu_new = Tmu_floor;
    }
    // Abundances: rates at T^{n+1} = mu^n T_mu^{n+1} with x^n, x_e^n frozen, x_H = 1 - 2x_H2
    // - x_H+ substituted, backward Euler on X' = A X + b solved in closed form.
    R Tn1 = mu * Tmu_new;
    R lnT1 = log(Tn1);
    R psi1 = P.G0 * sqrt(Tn1) / rmax(q.xe * P.n, R(1e-30)) + R(50.0);
    HRates<R> r = h_rates(c, p, P, Tn1, lnT1, xH2, xHp, q.xe, psi1);
    R kn = r.kgr * P.n;
    R DH2 = R(1.65) * r.zcrH2 + P.zpd + P.zpiH2 + r.zcd;
    R I = P.zpiH + r.zcrH + r.zci;
    R Rr = r.arr * q.xe * P.n + r.agr * P.n;
    // (I - A dt) X' = X + b dt with A = [[-(2kn+D), -kn], [-2I, -(I+R)]], b = (kn, I),
    // solved by Cramer's rule.  With a = 2kn + D and c = I + R the determinant and the
    // two numerators expand to sums of non-negative terms:
    //   det = 1 + (a + c) dt + (2 kn R + D c) dt^2
    //   num_H2 = x_H2 (1 + c dt) + kn dt (1 - x_H+ + R dt)
    //   num_H+ = x_H+ (1 + a dt) + I dt (1 - 2 x_H2 + D dt)
    // (algebraically identical to m22 r1 - m12 r2 etc., but free of the cancellation of
    // two large products when I dt >> 1), which also shows X' >= 0.
    R a = R(2.0) * kn + DH2;
    R cc = I + Rr;
    R det = R(1.0) + (a + cc) * dts + (R(2.0) * kn * Rr + DH2 * cc) * dts * dts;
    R num2 = xH2 * (R(1.0) + cc * dts) + kn * dts * ((R(1.0) - xHp) + Rr * dts);
    R nump = xHp * (R(1.0) + a * dts) + I * dts * ((R(1.0) - R(2.0) * xH2) + DH2 * dts);
    xH2 = num2 / det;
    xHp = nump / det;
    Tmu = Tmu_new;
    // Re-equilibrate C/O/e at (T^{n+1}, X^{n+1}) and update mu.
    q = equilibrium(c, P, Tn1, xH2, xHp);
    mu = mu_of(P, q.xe, xH2);
    ++nsub;
    if (last) { t = dtR; done = true; } else { t = t + dts; }
    if (!finite_(Tmu) || !finite_(xH2) || !finite_(xHp)) { status |= ST_NONFINITE; break; }
  }
  out.T = double(mu * Tmu);
  out.xH2 = double(xH2);
  out.xHp = double(xHp);
  out.xe = double(q.xe);
  out.xCp = double(q.xCp);
  out.xCO = double(q.xCO);
  out.nsub = nsub;
  out.status = status;
  out.newton_iters = 0;
  return out;
}

// ------------------------------------------------------------------ mode B: coupled implicit
// The paper (Sec. 6.1) names advancing Eqs. e:ODE1-e:ODE2 together with an iterative
// implicit scheme as the alternative to its sequential update.  READING: backward Euler
// on y = (T_mu, x_H2, x_H+), f(y) = (H/K, C_H2, C_H+), with T = mu^n T_mu (mu frozen at the
// substep start, as in the paper's scheme) and the C/O/e equilibrium and T_d re-solved
// inside every evaluation of f; same substep rule as mode A.
template <class R> inline void f_coupled(const CellIn& c, const Params& p, const Pre<R>& P, R mu, const R* y, R* f) {
  R T = mu * y[0];
  Equil<R> q = equilibrium(c, P, T, y[1], y[2]);
  Source<R> s = source_terms(c, p, P, T, y[1], y[2], q, R(-1.0));
  f[0] = (p.flags & F_FREEZE_T) ? R(0.0) : s.H / P.K;
  f[1] = s.CH2;
  f[2] = s.CHp;
}

// Solves the 3x3 system J d = b by Gaussian elimination with partial pivoting.
template <class R> inline bool solve3(R J[3][3], R b[3], R d[3]) {
  for (int k = 0; k < 3; ++k) {
    int piv = k;
    R best = rabs(J[k][k]);
    for (int i = k + 1; i < 3; ++i) {
      R v = rabs(J[i][k]);
      if (v > best) { best = v; piv = i; }
    }
    if (!(best > R(0.0))) return false;
    if (piv != k) {
      for (int j = 0; j < 3; ++j) { R tmp = J[k][j]; J[k][j] = J[piv][j]; J[piv][j] = tmp; }
      R tb = b[k]; b[k] = b[piv]; b[piv] = tb;
    }
    for (int i = k + 1; i < 3; ++i) {
      R m = J[i][k] / J[k][k];
      for (int j = k; j < 3; ++j) J[i][j] = J[i][j] - m * J[k][j];
      b[i] = b[i] - m * b[k];
    }
  }
  for (int i = 2; i >= 0; --i) {
    R s = b[i];
    for (int j = i + 1; j < 3; ++j) s = s - J[i][j] * d[j];
    d[i] = s / J[i][i];
  }
  return true;
}

// One backward-Euler substep y - y^n - dt f(y) = 0 by Newton's method with a forward-
// difference Jacobian (relative step 1e-7; abundance steps floored at 1e-17) and
// damping that keeps T_mu, x_H2, x_H+ and x_H positive (see below).  Converged
// when every full (undamped) step satisfies |d_i| <= rtol |y_i| (READING: relative for
// every component, so abundances as small as 1e-25 are still converged relatively).
// Returns the iteration count, or -1 on failure (also after maxit iterations).
template <class R> int newton_substep(const CellIn& c, const Params& p, const Pre<R>& P, R mu, const R* yn, R dts,
                                      const R* seed, R* y, int maxit) {
  for (int i = 0; i < 3; ++i) y[i] = seed[i];
  for (int it = 1; it <= maxit; ++it) {
    R f[3];
    f_coupled(c, p, P, mu, y, f);
    R J[3][3];
    for (int j = 0; j < 3; ++j) {
      R h = (j == 0) ? R(1e-7) * y[0] : rmax(R(1e-7) * rabs(y[j]), R(1e-17));
      R yp[3] = {y[0], y[1], y[2]};
      yp[j] = yp[j] + h;
      R fp[3];
      f_coupled(c, p, P, mu, yp, fp);
      for (int i = 0; i < 3; ++i) J[i][j] = ((i == j) ? R(1.0) : R(0.0)) - dts * (fp[i] - f[i]) / h;
    }
    R rhs[3];
    for (int i = 0; i < 3; ++i) rhs[i] = R(0.0) - (y[i] - yn[i] - dts * f[i]);
    R d[3];
    if (!solve3(J, rhs, d)) return -1;
    // Damping (READING; the root is unchanged, only the path to it), by blocks:
    //  - T_mu takes the step length lamT that keeps it at >= 1% of its value;
    //  - x_H2 and x_H+ share a step length lamX that keeps them and
    //    x_H = 1 - 2 x_H2 - x_H+ at >= 1% of their values (fraction 0.99 to the
    //    boundary), so that an abundance pressed against its bound does not freeze
    //    the temperature, nor the temperature the abundances;
    //  - if the x_H bound alone would cut the abundance step below 1% of its length
    //    (x_H -> 0 with the step pointing further down), the abundance step is instead
    //    projected onto that bound (the smallest change along the bound's normal
    //    (-2, -1)), which lets the iteration slide along it instead of stalling;
    //  - an abundance whose step is below 1e-8 in absolute terms cannot matter to the
    //    other unknowns: it does not limit lamX and is kept at >= 1% of its value on
    //    its own, so that a trace species driven towards zero does not freeze the rest.
    // Converged when no limit acted and every step is below newton_rtol |y_i|.
    R lamT = R(1.0);
    if (d[0] < R(0.0)) {
      R cap = R(0.99) * y[0] / (R(0.0) - d[0]);
      if (cap < lamT) lamT = cap;
    }
    R lamX = R(1.0);
    bool tiny[3] = {false, false, false};
    for (int i = 1; i < 3; ++i) {
      tiny[i] = !(rabs(d[i]) > R(1e-8));
      if (d[i] < R(0.0) && !tiny[i]) {
        R cap = R(0.99) * y[i] / (R(0.0) - d[i]);
        if (cap < lamX) lamX = cap;
      }
    }
    R xH = R(1.0) - R(2.0) * y[1] - y[2];
    R dxH = R(0.0) - R(2.0) * d[1] - d[2];
    bool proj = false;
    if (dxH < R(0.0)) {
      R cap = R(0.99) * rmax(xH, R(0.0)) / (R(0.0) - dxH);
      if (cap < R(0.01)) {
        R lim = R(0.0) - R(0.99) * rmax(xH, R(0.0));
        R beta = (dxH - lim) / R(5.0);
        d[1] = d[1] + R(2.0) * beta;
        d[2] = d[2] + beta;
        proj = true;
        lamX = R(1.0);
        for (int i = 1; i < 3; ++i) {
          tiny[i] = !(rabs(d[i]) > R(1e-8));
          if (d[i] < R(0.0) && !tiny[i]) {
            R c2 = R(0.99) * y[i] / (R(0.0) - d[i]);
            if (c2 < lamX) lamX = c2;
          }
        }
      } else if (cap < lamX) {
        lamX = cap;
      }
    }
    bool conv = !(lamT < R(1.0)) && !(lamX < R(1.0)) && !proj;
    for (int i = 0; i < 3; ++i) {
      R st = ((i == 0) ? lamT : lamX) * d[i];
      if (tiny[i] && y[i] + st < R(0.01) * y[i]) {
        st = R(0.0) - R(0.99) * y[i];
        conv = false;
      }
      R yi = y[i] + st;
      R step = yi - y[i];
      y[i] = yi;
      R tol = R(p.newton_rtol) * rabs(y[i]) + R(1e-300);
      if (rabs(step) > tol) conv = false;
    }
    if (!finite_(y[0]) || !finite_(y[1]) || !finite_(y[2])) return -1;
    if (conv) return it;
  }
  return -1;
}

// READING (Sec. 6.1 names the coupled implicit scheme but gives no solver for it): start
// point for a substep whose Newton iteration from the start state fails.  In hot gas
// where H is ionised as fast as H2 dissociation frees it, the root lies next to the
// x_H = 0 boundary, and the Newton direction at the start state points far outside
// the admissible region; the damped iteration then stalls in the corner x_H -> 0.
// The predictor sweeps the same backward-Euler equations block by block:
//  - abundances: the closed-form 2x2 backward Euler of the paper's own scheme (Eqs.
//    e:HH, e:HII with x_H = 1 - 2 x_H2 - x_H+), with every rate evaluated at the
//    current iterate (T, x, and x_e of the C/O/e equilibrium there); its numerators and
//    determinant are sums of non-negative terms, so x_H2, x_H+ and x_H stay >= 0;
//  - T_mu: one Newton step on its own equation g = T_mu - T_mu^n - dt H(T_mu, x)/K = 0
//    at the new abundances (forward-difference slope, relative step 1e-7); when
//    dg/dT_mu < 0.1 the explicit value T_mu^n + dt H/K is taken instead; the new T_mu is
//    kept within a factor 2 of the old.
// The sweeps stop when every component changed by less than 1e-3 relative (abundance
// changes relative to max(x, 1e-6)), or after 50 sweeps.  Newton then starts from this
// point; the equations, and so the root, are those of the plain iteration.
template <class R> void picard_predictor(const CellIn& c, const Params& p, const Pre<R>& P, R mu, const R* yn, R dts,
                                         R* y) {
  using std::log; using std::sqrt;
  for (int i = 0; i < 3; ++i) y[i] = yn[i];
  for (int k = 0; k < 50; ++k) {
    R T = mu * y[0];
    Equil<R> q = equilibrium(c, P, T, y[1], y[2]);
    R psi = P.G0 * sqrt(T) / rmax(q.xe * P.n, R(1e-30)) + R(50.0);
    HRates<R> r = h_rates(c, p, P, T, log(T), y[1], y[2], q.xe, psi);
    R kn = r.kgr * P.n;
    R DH2 = R(1.65) * r.zcrH2 + P.zpd + P.zpiH2 + r.zcd;
    R I = P.zpiH + r.zcrH + r.zci;
    R Rr = r.arr * q.xe * P.n + r.agr * P.n;
    R a = R(2.0) * kn + DH2;
    R cc = I + Rr;
    R det = R(1.0) + (a + cc) * dts + (R(2.0) * kn * Rr + DH2 * cc) * dts * dts;
    R x2 = (yn[1] * (R(1.0) + cc * dts) + kn * dts * ((R(1.0) - yn[2]) + Rr * dts)) / det;
    R xp = (yn[2] * (R(1.0) + a * dts) + I * dts * ((R(1.0) - R(2.0) * yn[1]) + DH2 * dts)) / det;
    R Tm = y[0];
    if (!(p.flags & F_FREEZE_T)) {
      R h = R(1e-7) * y[0];
      R ya[3] = {y[0], x2, xp}, yb[3] = {y[0] + h, x2, xp};
      R fa[3], fb[3];
      f_coupled(c, p, P, mu, ya, fa);
      f_coupled(c, p, P, mu, yb, fb);
      R g = y[0] - yn[0] - dts * fa[0];
      R gp = R(1.0) - dts * (fb[0] - fa[0]) / h;
      Tm = (gp > R(0.1)) ? y[0] - g / gp : yn[0] + dts * fa[0];
      Tm = rmin(rmax(Tm, R(0.5) * y[0]), R(2.0) * y[0]);
    }
    R ch = rabs(Tm - y[0]) / y[0];
    ch = rmax(ch, rabs(x2 - y[1]) / rmax(y[1], R(1e-6)));
    ch = rmax(ch, rabs(xp - y[2]) / rmax(y[2], R(1e-6)));
    y[0] = Tm;
    y[1] = x2;
    y[2] = xp;
    if (!finite_(y[0]) || !finite_(y[1]) || !finite_(y[2])) return;
    if (ch < R(1e-3)) return;
  }
}

// One substep's Newton solve: from the start state (at most newton_max iterations); if
// that fails, from the predictor above, with RESCUE_ITER_FACTOR times as many
// iterations (READING, same as for the predictor: in thermally unstable substeps the
// damped iteration can crawl to the root, up to ~300 iterations measured, and the
// alternative, halving the substep, changes the substep grid).  Returns the iterations
// of the successful solve, or -1; `pred` is set when the predictor was used.
constexpr int RESCUE_ITER_FACTOR = 8;
template <class R> int solve_substep(const CellIn& c, const Params& p, const Pre<R>& P, R mu, const R* yn, R dts,
                                     R* y, bool& pred) {
  if (!(p.flags & F_PREDICTOR)) {
    int it = newton_substep(c, p, P, mu, yn, dts, yn, y, p.newton_max);
    if (it >= 0) return it;
  }
  pred = true;
  R ys[3];
  picard_predictor(c, p, P, mu, yn, dts, ys);
  if (!finite_(ys[0]) || !finite_(ys[1]) || !finite_(ys[2])) return -1;
  return newton_substep(c, p, P, mu, yn, dts, ys, y, RESCUE_ITER_FACTOR * p.newton_max);
}

template <class R> CellOut step_coupled(const CellIn& c, const Params& p, double T_in, double xH2_in, double xHp_in,
                                        double dt) {
  CellOut out{};
  const Pre<R> P = prepare<R>(c, p);
  R xH2 = R(xH2_in), xHp = R(xHp_in);
  Equil<R> q = equilibrium(c, P, R(T_in), xH2, xHp);
  R mu = mu_of(P, q.xe, xH2);
  R Tmu = R(T_in) / mu;
  R t = R(0.0);
  int nsub = 0, status = ST_OK, iters = 0;
  const R dtR = R(dt);
  bool done = !(dt > 0.0);
  while (!done) {
    if (nsub >= p.max_substeps) { status |= ST_MAX_SUBSTEPS; break; }
    R T = mu * Tmu;
    R e = P.K * Tmu;
    Source<R> s = source_terms(c, p, P, T, xH2, xHp, q, R(-1.0));
    bool last;
    R dts = substep_length(p, dtR - t, e, (p.flags & F_FREEZE_T) ? R(0.0) : s.H, s.CH2, s.CHp, last);
    R yn[3] = {Tmu, xH2, xHp};
    R y[3];
    bool pred = false;
    int it = solve_substep(c, p, P, mu, yn, dts, y, pred);
    // READING: a substep whose Newton iteration fails from both start points is retried
    // at half length, up to 30 times; the cell is flagged ST_NEWTON.
    int halv = 0;
    while (it < 0 && halv < 30) {
      status |= ST_NEWTON;
      dts = dts * R(0.5);
      last = false;
      ++halv;
      it = solve_substep(c, p, P, mu, yn, dts, y, pred);
    }
    if (pred) status |= ST_PREDICTOR;
    if (it < 0) { status |= ST_NONFINITE; break; }
    iters += it;
    Tmu = rmax(y[0], R(p.T_floor) / mu);
    xH2 = y[1];
    xHp = y[2];
    q = equilibrium(c, P, mu * Tmu, xH2, xHp);
    mu = mu_of(P, q.xe, xH2);
    ++nsub;
    if (last) { t = dtR; done = true; } else { t = t + dts; }
    if (!finite_(Tmu) || !finite_(xH2) || !finite_(xHp)) { status |= ST_NONFINITE; break; }
  }
  out.T = double(mu * Tmu);
  out.xH2 = double(xH2);
  out.xHp = double(xHp);
  out.xe = double(q.xe);
  out.xCp = double(q.xCp);
  out.xCO = double(q.xCO);
  out.nsub = nsub;
  out.status = status;
  out.newton_iters = iters;
  return out;
}

}  // namespace oracle
