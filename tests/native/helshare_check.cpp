// Host check of the helicity-shared layout (helshare.h): for every process
// given on the command line, the diagram amplitudes of every summed helicity
// combination are evaluated twice in FP64 with the same vertex functions --
// once per combination through the program's wavefunction slots (the
// per-lane interpreter's order) and once through the helicity-shared variant
// arena (each produced wavefunction evaluated once per helicity pattern of its
// legs, inputs read from the variant the combination selects) -- and must
// agree bit for bit.  A block released before its last read, an overlap of
// live blocks, a wrong leg set or a wrong bit extraction changes some
// amplitude.  Inputs are random: external wavefunctions per (leg, helicity),
// leg momenta and the mask rows formed from them.  Also checks that every
// block lies inside the arena.  The split layout (prologue values once per
// helicity pattern, level by level; the rest per combination with one
// transient current) is checked the same way.  Prints per process: name,
// amplitudes compared, mismatches, arena variants, and the same for the split
// layout (area variants; -1 for processes of 4 legs), and for the per-lane
// evaluation with register forwarding (skipped stores poisoned); exit status
// 1 on any mismatch.
#define MEA_HD inline
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "generator.h"
#include "heget.cuh"
#include "helshare.h"

using namespace mea;

static uint32_t pext(uint32_t x, uint32_t S) {
  uint32_t r = 0;
  int k = 0;
  for (int l = 0; l < 8; ++l)
    if (S >> l & 1u) {
      if (x >> l & 1u) r |= 1u << k;
      ++k;
    }
  return r;
}
static uint32_t pdep(uint32_t v, uint32_t S) {
  uint32_t r = 0;
  int k = 0;
  for (int l = 0; l < 8; ++l)
    if (S >> l & 1u) {
      if (v >> k & 1u) r |= 1u << l;
      ++k;
    }
  return r;
}

struct Inputs {
  std::vector<std::vector<W4<double>>> ext;  // [leg][lambda bit]
  std::vector<double> mt;
};

// Value of a slot-producing op from its inputs x (ext: lam's bit of its leg).
static W4<double> produce(const Op& op, const W4<double>* x, const Inputs& in, uint32_t lam) {
  const double g = 1.1, gg = g * g;
  const double* M = in.mt.data();
  switch (op.type) {
    case OP_EXT: return in.ext[op.leg][lam >> op.leg & 1u];
    case OP_JVV: return jvv<double>(x[0], x[1], M + 5 * op.min[0], M + 5 * op.min[1], M[5 * op.mout + 4], g);
    case OP_JGGG: return jggg<double>(x[0], x[1], x[2], M[5 * op.mout + 4], gg);
    case OP_FVI: return fvi<double>(x[0], x[1], M + 5 * op.mout, M[5 * op.mout + 4], g);
    case OP_FVO: return fvo<double>(x[0], x[1], M + 5 * op.mout, M[5 * op.mout + 4], g);
    case OP_JIO: return jio<double>(x[0], x[1], M[5 * op.mout + 4], g);
    case OP_PVVV: return vvv_part<double>(x[0], x[1], M + 5 * op.min[0], M + 5 * op.min[1], M + 5 * op.min[2], g);
    case OP_PGGGG: return gggg_part<double>(x[0], x[1], x[2], gg);
    case OP_PIOV:
      return op.leg == 0 ? iov_part_i<double>(x[0], x[1], g)
                         : (op.leg == 1 ? iov_part_o<double>(x[0], x[1], g) : iov_part_v<double>(x[0], x[1], g));
  }
  std::fprintf(stderr, "unknown op %d\n", op.type);
  std::exit(2);
}
static cx<double> amplitude(const Op& op, const W4<double>* x, const Inputs& in) {
  const double g = 1.1, gg = g * g;
  const double* M = in.mt.data();
  switch (op.type) {
    case OP_AVVV: return vvv_amp<double>(x[0], x[1], x[2], M + 5 * op.min[0], M + 5 * op.min[1], M + 5 * op.min[2], g);
    case OP_AGGGG: return gggg_amp<double>(x[0], x[1], x[2], x[3], gg);
    case OP_AIOV: return iov_amp<double>(x[0], x[1], x[2], g);
    case OP_ADOT: return part_contract<double>(x[0], x[1], (op.leg & 1u) != 0, (op.leg & 2u) != 0);
  }
  std::fprintf(stderr, "unknown amplitude op %d\n", op.type);
  std::exit(2);
}

int main(int argc, char** argv) {
  int bad = 0;
  // --all: every one of the 2^n_ext helicity combinations (the full helicity
  // sum), not only those the selection rules keep
  bool all = false;
  for (int a = 1; a < argc; ++a) {
    if (std::string(argv[a]) == "--all") {
      all = true;
      continue;
    }
    std::vector<int> pdg;
    std::string s = argv[a];
    for (size_t p = 0; p < s.size();) {
      size_t e = s.find(',', p);
      if (e == std::string::npos) e = s.size();
      pdg.push_back(std::atoi(s.substr(p, e - p).c_str()));
      p = e + 1;
    }
    const Program P = build_program(pdg);
    const HsProgram Q = build_helicity_shared(P, P.n_hel);
    const int n_ops = (int)P.ops.size();
    std::mt19937_64 rng(0x5eed + a);
    auto u = [&]() { return std::uniform_real_distribution<double>(-1.0, 1.0)(rng); };
    Inputs in;
    in.ext.assign(P.n_ext, std::vector<W4<double>>(2));
    for (auto& l : in.ext)
      for (auto& w : l)
        for (int k = 0; k < 4; ++k) w.c[k] = {u(), u()};
    std::vector<double> leg(4 * P.n_ext);
    for (double& x : leg) x = u();
    in.mt.assign(5 * P.masks.size(), 0.0);
    for (size_t r = 0; r < P.masks.size(); ++r) {
      double q[4] = {0, 0, 0, 0};
      for (int l = 0; l < P.n_ext; ++l)
        if (P.masks[r] >> l & 1u)
          for (int m = 0; m < 4; ++m) q[m] += leg[4 * l + m];
      for (int m = 0; m < 4; ++m) in.mt[5 * r + m] = q[m];
      in.mt[5 * r + 4] = 1.0 / (q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3]);
    }
    const int n_hel = all ? (1 << P.n_ext) : P.n_hel;
    const std::vector<int8_t>& hel = all ? P.hel_all : P.hel;
    std::vector<uint32_t> lam(n_hel);
    for (int h = 0; h < n_hel; ++h)
      for (int l = 0; l < P.n_ext; ++l)
        if (hel[h * P.n_ext + l] > 0) lam[h] |= 1u << l;

    // per combination through the slots
    std::vector<cx<double>> ref((size_t)n_hel * P.n_diagrams);
    for (int h = 0; h < n_hel; ++h) {
      std::vector<W4<double>> slots(P.n_slots);
      int d = 0;
      for (const Op& op : P.ops) {
        W4<double> x[4];
        const int n_in = op.type == OP_EXT ? 0 : op.n_in;
        for (int k = 0; k < n_in; ++k) x[k] = slots[op.in[k]];
        if (is_amp_op(op.type)) ref[(size_t)h * P.n_diagrams + d++] = amplitude(op, x, in);
        else slots[op.out] = produce(op, x, in, lam[h]);
      }
    }
    // helicity shared through the arena
    std::vector<W4<double>> arena(Q.arena);
    int64_t compared = 0, mismatched = 0;
    int d = 0;
    for (int i = 0; i < n_ops; ++i) {
      const Op& op = P.ops[i];
      const HsOp& q = Q.ops[i];
      const int n_in = op.type == OP_EXT ? 0 : op.n_in;
      for (int k = 0; k < n_in; ++k)
        if (q.in_off[k] + (1 << __builtin_popcount(q.in_mask[k])) > Q.arena) {
          std::printf("input block outside the arena at op %d\n", i);
          bad = 1;
        }
      if (!is_amp_op(op.type)) {
        const int nv = 1 << __builtin_popcount(q.out_mask);
        if (q.out_off + nv > Q.arena) {
          std::printf("output block outside the arena at op %d\n", i);
          bad = 1;
          continue;
        }
        for (int k = 0; k < n_in; ++k) {  // the lanes of one op write while others still read
          const int lo = q.in_off[k], hi = lo + (1 << __builtin_popcount(q.in_mask[k]));
          if (q.out_off < hi && lo < q.out_off + nv) {
            std::printf("output block overlaps input %d at op %d\n", k, i);
            bad = 1;
          }
        }
        for (int v = 0; v < nv; ++v) {
          const uint32_t lf = pdep((uint32_t)v, q.out_mask);
          W4<double> x[4];
          for (int k = 0; k < n_in; ++k) x[k] = arena[q.in_off[k] + pext(lf, q.in_mask[k])];
          arena[q.out_off + v] = produce(op, x, in, lf);
        }
      } else {
        for (int h = 0; h < n_hel; ++h) {
          W4<double> x[4];
          for (int k = 0; k < n_in; ++k) x[k] = arena[q.in_off[k] + pext(lam[h], q.in_mask[k])];
          const cx<double> z = amplitude(op, x, in);
          const cx<double>& r = ref[(size_t)h * P.n_diagrams + d];
          ++compared;
          if (std::memcmp(&z, &r, sizeof(z)) != 0) ++mismatched;
        }
        ++d;
      }
    }
    // split: prologue values once per helicity pattern, level by level; the
    // rest per combination with the transient current held aside
    int64_t split_compared = 0, split_mismatched = 0;
    int split_area = -1;
    if (P.n_ext >= 5) {
      const HsSplitProgram S = build_split_shared(P, P.n_hel);
      split_area = S.area;
      std::vector<W4<double>> area(S.area);
      for (size_t t = 0; t < S.tasks.size(); ++t) {
        const int i = (int)(S.tasks[t] >> 8), v = (int)(S.tasks[t] & 0xffu);
        const Op& op = P.ops[i];
        const HsOp& q = S.rec[i];
        const uint32_t lf = pdep((uint32_t)v, q.out_mask);
        W4<double> x[4];
        const int n_in = op.type == OP_EXT ? 0 : op.n_in;
        for (int k = 0; k < n_in; ++k) {
          if (q.in_off[k] == kHsTransient) { std::printf("prologue input is transient\n"); bad = 1; continue; }
          x[k] = area[q.in_off[k] + pext(lf, q.in_mask[k])];
        }
        if (q.out_off + (1 << __builtin_popcount(q.out_mask)) > S.area) { std::printf("prologue block outside\n"); bad = 1; continue; }
        area[q.out_off + v] = produce(op, x, in, lf);
      }
      for (int h = 0; h < n_hel; ++h) {
        W4<double> tr;
        int dd = 0;
        for (size_t j = 0; j < S.main_ops.size(); ++j) {
          const Op& op = S.main_ops[j];
          const HsOp& q = S.main_rec[j];
          W4<double> x[4];
          for (int k = 0; k < op.n_in; ++k)
            x[k] = q.in_off[k] == kHsTransient ? tr : area[q.in_off[k] + pext(lam[h], q.in_mask[k])];
          if (is_amp_op(op.type)) {
            const cx<double> z = amplitude(op, x, in);
            const cx<double>& r = ref[(size_t)h * P.n_diagrams + dd++];
            ++split_compared;
            if (std::memcmp(&z, &r, sizeof(z)) != 0) ++split_mismatched;
          } else {
            tr = produce(op, x, in, lam[h]);
          }
        }
        if (dd != P.n_diagrams) { std::printf("split: %d amplitudes, %d diagrams\n", dd, P.n_diagrams); bad = 1; }
      }
    }
    // per combination through the slots with register forwarding: a skipped
    // store leaves its slot poisoned (NaN), so a read of it anywhere but from
    // the register changes the amplitude
    int64_t fwd_compared = 0, fwd_mismatched = 0;
    {
      const std::vector<uint8_t> fw = build_forwarding_flags(P);
      const double qnan = std::nan("");
      for (int h = 0; h < n_hel; ++h) {
        std::vector<W4<double>> slots(P.n_slots);
        for (auto& w : slots)
          for (int k = 0; k < 4; ++k) w.c[k] = {qnan, qnan};
        W4<double> last;
        for (int k = 0; k < 4; ++k) last.c[k] = {qnan, qnan};
        int dd = 0;
        for (int i = 0; i < n_ops; ++i) {
          const Op& op = P.ops[i];
          W4<double> x[4];
          const int n_in = op.type == OP_EXT ? 0 : op.n_in;
          for (int k = 0; k < n_in; ++k) x[k] = (fw[i] >> k & 1u) ? last : slots[op.in[k]];
          if (is_amp_op(op.type)) {
            const cx<double> z = amplitude(op, x, in);
            const cx<double>& r = ref[(size_t)h * P.n_diagrams + dd++];
            ++fwd_compared;
            if (std::memcmp(&z, &r, sizeof(z)) != 0) ++fwd_mismatched;
          } else {
            last = produce(op, x, in, lam[h]);
            if (!(fw[i] & 16u)) slots[op.out] = last;
          }
        }
      }
    }
    if (mismatched || split_mismatched || fwd_mismatched) bad = 1;
    std::printf("%s %lld %lld %d %lld %lld %d %lld %lld\n", argv[a], (long long)compared, (long long)mismatched, Q.arena,
                (long long)split_compared, (long long)split_mismatched, split_area, (long long)fwd_compared,
                (long long)fwd_mismatched);
  }
  return bad;
}
