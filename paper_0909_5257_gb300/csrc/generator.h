// Process generator: from a list of partons to the per-(event, helicity)
// program that the CUDA amplitude kernels execute.
//
// For a process it builds
//   * the graph of off-shell currents shared between Feynman diagrams
//     (HELAS-style: each current is one call of jvvxx0 / jgggx0 / a qqg current
//     function, Sec. 4 of arXiv:0909.5257) and one amplitude operation per
//     diagram (vvvxxx, ggggxx, iovxx0), so that the diagram count equals
//     Table 1;
//   * for every amplitude its colour coefficients on the Table 1 colour basis
//     (single traces for gluons, Eq. (color-basis); strings for one quark line;
//     two strings joined by one exchanged gluon for two quark lines);
//   * the exact colour matrix N = K / D of Eq. (color-matrix), K integer;
//   * the helicity combinations allowed by the massless selection rules;
//   * vertex partials: diagram amplitudes whose amplitude vertex shares all
//     inputs but one are evaluated as contractions of that input with the
//     shared partial vertex (heget.cuh, "vertex partials");
//   * an evaluation order with wavefunction-slot reuse.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mea {

enum OpType : uint8_t {
  OP_EXT = 1,    // external wavefunction of leg in[0]
  OP_JVV = 2,    // gluon current from gluons in[0], in[1] (jvvxx0)
  OP_JGGG = 3,   // gluon current from gluons in[0..2] in call order (jgggx0)
  OP_FVI = 4,    // off-shell quark current from quark in[0] and gluon in[1]
  OP_FVO = 5,    // off-shell antiquark current from in[0] (barred) and gluon in[1]
  OP_JIO = 6,    // gluon current from quark in[0] and barred quark in[1]
  OP_AVVV = 7,   // amplitude vvvxxx(in[0], in[1], in[2])
  OP_AGGGG = 8,  // amplitude ggggxx(in[0..3]) in call order
  OP_AIOV = 9,   // amplitude iovxx0(fi = in[0], fo = in[1], v = in[2])
  OP_ADOT = 10,  // amplitude: free wavefunction in[0] contracted with the vertex partial in[1];
                 // leg bit 0: plain (spinor) instead of metric contraction, bit 1: negate
  OP_PVVV = 11,  // vertex partial of vvvxxx with a free first argument: in[0], in[1] the other two,
                 // min[0] the free argument's row, min[1], min[2] those of in[0], in[1]
  OP_PGGGG = 12, // vertex partial G(in[0], in[1], in[2]) of ggggxx (heget.cuh gggg_part)
  OP_PIOV = 13,  // vertex partial of iovxx0, leg = free argument (0 fi, 1 fo, 2 V):
                 // (fo, V), (fi, V) or (fi, fo) in in[0], in[1]
};

// Amplitude operations (one per Feynman diagram, in diagram-ordinal order).
inline bool is_amp_op(int t) { return t == OP_AVVV || t == OP_AGGGG || t == OP_AIOV || t == OP_ADOT; }
// Vertex partials: like currents they fill a wavefunction slot.
inline bool is_partial_op(int t) { return t >= OP_PVVV && t <= OP_PIOV; }

// 32-byte operation record, read uniformly by every lane.
struct Op {
  uint8_t type;
  uint8_t n_in;
  uint16_t out;        // output slot (currents); diagram ordinal (amplitudes)
  uint16_t in[4];      // input slots
  uint16_t mout;       // mask-table row of the produced line (momentum, 1/P^2)
  uint16_t min[4];     // mask-table rows of the inputs
  uint16_t leg;        // OP_EXT: leg index
  uint32_t col_begin;  // amplitudes: first colour entry
  uint32_t col_count;  // amplitudes: number of colour entries
};
static_assert(sizeof(Op) == 32, "Op must stay 32 bytes");

// One colour coefficient: J[alpha] += (re + i im) * amplitude.
struct ColEntry {
  uint16_t alpha;
  int8_t re, im;
};

enum Family { FAM_GLUON = 0, FAM_ONE_LINE = 1, FAM_TWO_LINES = 2 };

struct Program {
  int n_ext = 0;
  std::vector<int> pdg;
  std::vector<int> incoming;          // 1 for legs 0,1
  std::vector<int> leg_type;          // 0 gluon, 1 quark-type wavefunction u/v (psi), 2 barred (psibar)
  std::vector<int> leg_is_quark;      // 1 quark, 0 antiquark (for spinor choice)
  Family family = FAM_GLUON;
  int root = 0;
  std::vector<Op> ops;
  std::vector<ColEntry> col;
  std::vector<uint32_t> masks;        // bit patterns of the mask-table rows
  int n_slots = 0;
  int n_diagrams = 0;
  int n_currents = 0;
  int n_partials = 0;                 // vertex partials shared by several diagram amplitudes
  int n_colour = 0;                   // colour basis size (Table 1)
  int n_a = 1, n_b = 1;
  std::vector<int64_t> cf_num;        // [m*m] exact colour matrix K of the basis, N = K / cf_den
  int64_t cf_den = 1;
  int64_t cf_max_abs = 0;
  // Colour amplitudes the kernels accumulate.  For pure-gluon processes the
  // reflection identity J_rev(a) = (-1)^n J_a (checked on every diagram's
  // coefficients) halves them: only canonical orderings are kept and the
  // colour matrix is folded, K'_ab = 2 (K_ab + (-1)^n K_a,rev(b)).  Otherwise
  // n_jamp = n_colour and cf_jamp = cf_num.
  int n_jamp = 0;
  std::vector<int64_t> cf_jamp;       // [n_jamp * n_jamp], same denominator cf_den
  int64_t cf_jamp_max_abs = 0;
  std::vector<int8_t> hel;            // [n_hel][n_ext], physical helicities
  int n_hel = 0;
  std::vector<int8_t> hel_all;        // [2^n_ext][n_ext]
  double flops_per_hel = 0;
  double flops_per_hel_plain = 0;     // the same with one vertex call per diagram
  std::string basis_text;             // human-readable basis (debug)
};

struct BuildOptions {
  // false: every diagram amplitude is its own vertex call (no shared partials)
  bool vertex_partials = true;
  // schedule: false keeps the order with fewer live wavefunction slots (the
  // interpreter's memory traffic); true keeps each partial's diagrams together
  // (shorter live ranges in the straight-line kernels' registers)
  bool group_together = false;
};

// Throws std::runtime_error on unsupported input.  The diagram amplitudes and
// their colour coefficients do not depend on the options; their order and the
// rounding of the amplitudes do.
Program build_program(const std::vector<int>& pdg, const BuildOptions& opt = BuildOptions());

// Distinct signed non-zero values of the upper triangle of K (Table 5 count).
int count_unique_colour_values(const Program& p);

// Algorithmic real-FLOP cost of one operation (colour entries not included).
double op_flop_cost(const Op& op);

}  // namespace mea
