// Helicity-shared evaluation of a process program.
//
// Every wavefunction the program produces (external state, off-shell current,
// vertex partial) depends on the helicities of the external legs that flow
// into it and on nothing else of the helicity combination.  The per-lane
// interpreter evaluates it once per (event, helicity) lane; here it is
// evaluated once per distinct helicity pattern of its own legs ("variant"):
// a current of k legs has 2^k variants, however many of the summed
// helicity combinations share each.  Diagram amplitudes depend on every leg
// and are still evaluated once per summed combination.  The values are the
// same operations on the same inputs, so every amplitude is bit-identical to
// the per-lane interpreter's.
//
// Storage: per event, an arena of 32-byte FP32 wavefunction variants.  The
// produced value of leg set S occupies 2^|S| consecutive variants, variant v
// holding the helicity pattern whose i-th lowest leg of S has helicity +1
// exactly when bit i of v is set.  Blocks are allocated in program order and
// released after their last reader (never before the reading op's own output
// is placed, so an op's output never overlaps its inputs).
#pragma once
#include <cstdint>
#include <vector>

#include "generator.h"

namespace mea {

// 16-byte record parallel to Program::ops.
struct HsOp {
  uint16_t out_off;    // arena offset (variants) of the produced block (slot-producing ops)
  uint16_t in_off[4];  // arena offsets of the inputs' blocks
  uint8_t out_mask;    // legs of the produced wavefunction (bit l: leg l)
  uint8_t in_mask[4];  // legs of each input
  uint8_t pad;
};
static_assert(sizeof(HsOp) == 16, "HsOp must stay 16 bytes");

struct HsProgram {
  std::vector<HsOp> ops;
  int arena = 0;              // variants per event (the allocator's high-water mark)
  int64_t live_peak = 0;      // largest sum of live variants (no fragmentation)
  int64_t variants = 0;       // variant evaluations of slot-producing ops per event
  int64_t lane_copies = 0;    // the same ops evaluated once per helicity lane (H x ops)
  int64_t amp_lanes = 0;      // amplitude evaluations per event (H x diagrams)
  double flops_event = 0;     // FLOPs per event: variants and amplitude lanes x op cost
  double flops_event_lane = 0;  // the same for the per-lane interpreter (colour entries excluded)
  double lane_use = 0;        // variant evaluations / warp lanes issued for them (32-lane warps)
};

// Builds the helicity-shared layout of P for H summed helicity combinations.
// Throws std::runtime_error when the process has more than 8 legs or the
// arena exceeds 65535 variants.
HsProgram build_helicity_shared(const Program& P, int H);

// Split evaluation: the wavefunctions of at most n_ext - 3 legs (external
// states, the shorter currents and vertex partials, which the diagrams share
// and which stay live over most of the program) are evaluated once per
// helicity pattern of their legs in a prologue, level by level (level k: the
// values of k legs, whose inputs all have fewer); the rest of the program --
// the currents of n_ext - 2 legs, each read once by the very next op, and the
// diagram amplitudes -- runs once per (event, helicity) lane with that one
// transient current in registers.  Same operations on the same inputs as the
// per-lane program: bit-identical amplitudes.
constexpr uint16_t kHsTransient = 0xFFFFu;  // HsOp::in_off of an input held in registers

struct HsSplitProgram {
  int area = 0;                    // variants per event of the prologue values
  int levels = 0;                  // prologue levels (leg counts 1 .. levels)
  std::vector<uint32_t> tasks;     // prologue: (op index << 8) | variant, level by level
  std::vector<int> level_end;      // end of each level's tasks
  std::vector<HsOp> rec;           // per op of the program: prologue ops: output and input blocks;
                                   //   other ops: input blocks, kHsTransient for the transient
  std::vector<Op> main_ops;        // the per-lane ops in program order (transient currents, amplitudes)
  std::vector<HsOp> main_rec;      // their records
  int64_t prologue_variants = 0;
  double flops_event = 0;          // per event: prologue variants + H x per-lane ops, each at its cost
};

// Throws std::runtime_error when the program does not have that structure (a
// longer value read other than once by the next op) or the area exceeds 65535
// variants.
HsSplitProgram build_split_shared(const Program& P, int H);

// Register forwarding in the per-lane interpreter: per op, bit k (0..3) when
// input k is the output of the op just before (read from the register that
// holds it), bit 4 when the op's output is read by nothing but the next op
// (kept in that register only, never stored to its slot).
std::vector<uint8_t> build_forwarding_flags(const Program& P);

}  // namespace mea
