// Host program that runs the library's own step functions on the CPU, for tests that
// need no GPU (not part of libtc_gb300.so, and not reachable from the C ABI or the
// binding; built and run by tests/test_host_step.py with the library's csrc/ on the
// include path).  Each cell goes through the same
// sequence as one lane of k_step: load_cell, the initial C/O/e equilibrium that sets mu,
// substeps of the selected mode until the step's end (or the substep cap), store_cell.
// Only host code is executed: the device translation of this file is never launched.
//
// Usage: tc_hoststep IN OUT MODE dvdr T_cmb chi0 opt_over_fuv tau_ratio limiter fd_rel
//                    rtol rtol_mixed T_floor newton_max max_sub flags
//   MODE 0 (the paper's sequential scheme), 1 (coupled Newton, FP64), 2 (mixed).
//   IN:  n as int64, then 12 arrays of n doubles (n, chi_pe, chi_lw, f_shld_H2,
//        f_shld_C, F_LyC, xi, Z'_g, Z'_d, T, x_H2, x_H+), then dt as a double.
//   OUT: 6 arrays of n doubles (T, x_H2, x_H+, x_e, x_C+, x_CO), then 3 arrays of n
//        int32 (substeps, status bits, Newton iterations).
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tc_kernels.cuh"

using namespace tcg;

int main(int argc, char** argv) {
  if (argc != 17) {
    fprintf(stderr, "usage: %s IN OUT MODE <13 parameters>\n", argv[0]);
    return 2;
  }
  FILE* fh = fopen(argv[1], "rb");
  if (!fh) return 3;
  int64_t n = 0;
  if (fread(&n, 8, 1, fh) != 1 || n <= 0) return 4;
  std::vector<double> in(12 * (size_t)n);
  double dt = 0;
  if (fread(in.data(), 8, in.size(), fh) != in.size() || fread(&dt, 8, 1, fh) != 1) return 5;
  fclose(fh);
  const int mode = atoi(argv[3]);
  if (mode < 0 || mode > 2) return 6;
  DevParams p;
  p.dvdr_kms_pc = atof(argv[4]);
  p.T_cmb = atof(argv[5]);
  p.chi0 = atof(argv[6]);
  p.opt_over_fuv = atof(argv[7]);
  p.tau_ratio = atof(argv[8]);
  p.limiter = atof(argv[9]);
  p.fd_rel = atof(argv[10]);
  p.rtol = atof(argv[11]);
  p.rtol_mixed = atof(argv[12]);
  p.T_floor = atof(argv[13]);
  p.newton_max = atoi(argv[14]);
  p.max_sub = atoi(argv[15]);
  p.flags = (unsigned)strtoul(argv[16], nullptr, 10);

  std::vector<double> outd(6 * (size_t)n);
  std::vector<int> outi(3 * (size_t)n);
  auto col = [&](int k) { return in.data() + (size_t)k * n; };
  DevFields f{};
  f.n = col(0); f.chi_pe = col(1); f.chi_lw = col(2); f.fh2 = col(3); f.fc = col(4);
  f.Flyc = col(5); f.xi = col(6); f.Zg = col(7); f.Zd = col(8);
  f.T = col(9); f.xH2 = col(10); f.xHp = col(11);
  double* od = outd.data();
  int* oi = outi.data();
  for (int64_t i = 0; i < n; ++i) {
    CellC<double> c;
    double T0, x20, xp0;
    load_cell(f, i, p, c, T0, x20, xp0);
    LaneState s;
    s.t = 0.0; s.xH2 = x20; s.xHp = xp0; s.Td = -1.0; s.nsub = 0; s.status = 0; s.iters = 0;
    CellC<float> cf = cast_cell<float>(c);
    CellC<df64> cd = cast_cell<df64>(c);
    if (mode == 2) {  // the mixed kernels solve the initial equilibrium in df64
      ChemT<df64> b0 = chem_T(cd, df64(T0), p.flags);
      Equil<df64> q0 = equilibrium(cd, b0, df64(x20), df64(xp0), df64(-1.0));
      s.xe = double(q0.xe); s.xCp = double(q0.xCp); s.xCO = double(q0.xCO);
    } else {
      ChemT<double> b0 = chem_T(c, T0, p.flags);
      Equil<double> q0 = equilibrium(c, b0, x20, xp0, -1.0);
      s.xe = q0.xe; s.xCp = q0.xCp; s.xCO = q0.xCO;
    }
    double xe_g = s.xe, td_g = -1.0;
    df64 td_hp = df64(-1.0);
    float xe_gf = float(s.xe), td_gf = -1.f;
    s.mu = c.muH / (1.1 + s.xe - x20);
    s.Tmu = T0 / s.mu;
    while (s.t < dt) {
      if (s.nsub >= p.max_sub) {
        s.status |= ST_MAX_SUB;
        s.t = dt;
        break;
      }
      if (mode == 0) substep_paper(c, p, dt, s);
      else if (mode == 1) substep_newton64(c, p, dt, s, xe_g, td_g);
      else substep_mixed(c, cd, cf, p, dt, s, xe_gf, td_gf, td_hp);
      if (!finite3(s.Tmu, s.xH2, s.xHp)) {
        s.status |= ST_NONFIN;
        s.t = dt;
      }
    }
    DevFields o{};
    o.T = od; o.xH2 = od + n; o.xHp = od + 2 * n; o.xe = od + 3 * n; o.xCp = od + 4 * n; o.xCO = od + 5 * n;
    o.nsub = oi; o.status = oi + n; o.iters = oi + 2 * n;
    store_cell(o, i, s);
  }
  FILE* fo = fopen(argv[2], "wb");
  if (!fo) return 7;
  if (fwrite(outd.data(), 8, outd.size(), fo) != outd.size() || fwrite(outi.data(), 4, outi.size(), fo) != outi.size())
    return 8;
  fclose(fo);
  return 0;
}
