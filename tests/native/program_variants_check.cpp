// Host check of the process generator's schedules: the program built with
// shared vertex partials (in either schedule order) and the program with one
// vertex call per diagram compute the same colour amplitudes
// J_alpha = sum_d c_alpha,d A_d (Eq. (color-amplitude) of arXiv:0909.5257) and
// use the same mask table, which the straight-line kernels of every variant
// share with the runtime program.  Inputs are random: external wavefunctions,
// leg momenta, and the mask rows formed from them.  Prints the largest
// relative deviation per process; exit status 1 if a mask table differs.
#define MEA_HD inline
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "generator.h"
#include "heget.cuh"

using namespace mea;
typedef std::complex<double> Z;

static std::vector<Z> colour_amplitudes(const Program& P, uint64_t seed) {
  std::mt19937_64 rng(seed);
  auto u = [&]() { return std::uniform_real_distribution<double>(-1.0, 1.0)(rng); };
  std::vector<std::array<double, 4>> leg(P.n_ext);
  for (auto& l : leg)
    for (double& x : l) x = u();
  std::vector<double> mt(5 * P.masks.size());
  for (size_t r = 0; r < P.masks.size(); ++r) {
    double q[4] = {0, 0, 0, 0};
    for (int l = 0; l < P.n_ext; ++l)
      if (P.masks[r] >> l & 1u)
        for (int m = 0; m < 4; ++m) q[m] += leg[l][m];
    for (int m = 0; m < 4; ++m) mt[5 * r + m] = q[m];
    mt[5 * r + 4] = 1.0 / (q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3]);
  }
  std::vector<W4<double>> ext(P.n_ext);
  for (auto& w : ext)
    for (int k = 0; k < 4; ++k) w.c[k] = {u(), u()};
  std::vector<W4<double>> slots(P.n_slots);
  std::vector<Z> J(P.n_jamp);
  const double g = 1.1, gg = g * g;
  const double* M = mt.data();
  for (const Op& op : P.ops) {
    auto S = [&](int k) { return slots[op.in[k]]; };
    cx<double> a{0, 0};
    switch (op.type) {
      case OP_EXT: slots[op.out] = ext[op.leg]; continue;
      case OP_JVV: slots[op.out] = jvv<double>(S(0), S(1), M + 5 * op.min[0], M + 5 * op.min[1], M[5 * op.mout + 4], g); continue;
      case OP_JGGG: slots[op.out] = jggg<double>(S(0), S(1), S(2), M[5 * op.mout + 4], gg); continue;
      case OP_FVI: slots[op.out] = fvi<double>(S(0), S(1), M + 5 * op.mout, M[5 * op.mout + 4], g); continue;
      case OP_FVO: slots[op.out] = fvo<double>(S(0), S(1), M + 5 * op.mout, M[5 * op.mout + 4], g); continue;
      case OP_JIO: slots[op.out] = jio<double>(S(0), S(1), M[5 * op.mout + 4], g); continue;
      case OP_PVVV:
        slots[op.out] = vvv_part<double>(S(0), S(1), M + 5 * op.min[0], M + 5 * op.min[1], M + 5 * op.min[2], g);
        continue;
      case OP_PGGGG: slots[op.out] = gggg_part<double>(S(0), S(1), S(2), gg); continue;
      case OP_PIOV:
        slots[op.out] = op.leg == 0 ? iov_part_i<double>(S(0), S(1), g)
                                    : (op.leg == 1 ? iov_part_o<double>(S(0), S(1), g) : iov_part_v<double>(S(0), S(1), g));
        continue;
      case OP_AVVV: a = vvv_amp<double>(S(0), S(1), S(2), M + 5 * op.min[0], M + 5 * op.min[1], M + 5 * op.min[2], g); break;
      case OP_AGGGG: a = gggg_amp<double>(S(0), S(1), S(2), S(3), gg); break;
      case OP_AIOV: a = iov_amp<double>(S(0), S(1), S(2), g); break;
      case OP_ADOT: a = part_contract<double>(S(0), S(1), (op.leg & 1u) != 0, (op.leg & 2u) != 0); break;
      default: std::fprintf(stderr, "unknown op %d\n", op.type); std::exit(2);
    }
    for (uint32_t k = 0; k < op.col_count; ++k) {
      const ColEntry& c = P.col[op.col_begin + k];
      J[c.alpha] += Z(c.re, c.im) * Z(a.r, a.i);
    }
  }
  return J;
}

int main(int argc, char** argv) {
  int bad = 0;
  for (int i = 1; i < argc; ++i) {
    std::vector<int> pdg;
    std::string s = argv[i];
    for (size_t p = 0; p < s.size();) {
      size_t e = s.find(',', p);
      if (e == std::string::npos) e = s.size();
      pdg.push_back(std::atoi(s.substr(p, e - p).c_str()));
      p = e + 1;
    }
    BuildOptions fewest, grouped, plain;
    grouped.group_together = true;
    plain.vertex_partials = false;
    const Program A = build_program(pdg, fewest), B = build_program(pdg, grouped), C = build_program(pdg, plain);
    if (A.masks != B.masks || A.masks != C.masks || A.n_diagrams != C.n_diagrams) bad = 1;
    double worst = 0;
    for (uint64_t seed = 1; seed <= 8; ++seed) {
      const std::vector<Z> ja = colour_amplitudes(A, seed), jb = colour_amplitudes(B, seed), jc = colour_amplitudes(C, seed);
      double nrm = 0;
      for (const Z& z : jc) nrm = std::max(nrm, std::abs(z));
      for (size_t k = 0; k < jc.size(); ++k)
        worst = std::max(worst, std::max(std::abs(ja[k] - jc[k]), std::abs(jb[k] - jc[k])) / nrm);
    }
    std::printf("%s %.3e %d\n", argv[i], worst, A.n_partials);
  }
  return bad;
}
