// Helicity-shared layout of a process program (see helshare.h).
#include "helshare.h"

#include <stdexcept>
#include <string>

namespace mea {

HsProgram build_helicity_shared(const Program& P, int H) {
  if (P.n_ext > 8) throw std::runtime_error("helicity sharing: more than 8 legs");
  const int n_ops = (int)P.ops.size();
  HsProgram Q;
  Q.ops.assign(n_ops, HsOp{});

  // Pass 1: the producer (op index) of the value each input reads, the legs
  // of every produced value and the last op that reads it.
  std::vector<int> holder(P.n_slots, -1), last_read(n_ops, -1);
  std::vector<int> src(4 * (size_t)n_ops, -1);
  std::vector<uint32_t> legs(n_ops, 0);
  for (int i = 0; i < n_ops; ++i) {
    const Op& op = P.ops[i];
    const int n_in = op.type == OP_EXT ? 0 : op.n_in;
    uint32_t u = 0;
    for (int k = 0; k < n_in; ++k) {
      const int s = holder.at(op.in[k]);
      if (s < 0) throw std::runtime_error("helicity sharing: slot read before it is written");
      src[4 * (size_t)i + k] = s;
      last_read[s] = i;
      u |= legs[s];
    }
    if (!is_amp_op(op.type)) {
      legs[i] = op.type == OP_EXT ? (1u << op.leg) : u;
      if (op.type != OP_EXT && !is_partial_op(op.type) && legs[i] != P.masks.at(op.mout))
        throw std::runtime_error("helicity sharing: current legs differ from its momentum row");
      holder.at(op.out) = i;
    } else if (u != (1u << P.n_ext) - 1u) {
      throw std::runtime_error("helicity sharing: amplitude does not cover every leg");
    }
  }

  // Pass 2: arena blocks.  Power-of-two sizes, one free list per size; a new
  // block starts at a multiple of min(size, 4) variants (128 bytes), so that a
  // warp's accesses to a block are whole cache lines.  An op's output is placed
  // before the blocks of its last-read inputs are released.
  std::vector<std::vector<int>> free_list(10);
  int top = 0;
  int64_t live = 0;
  std::vector<int> off(n_ops, -1);
  double lanes_issued = 0;
  for (int i = 0; i < n_ops; ++i) {
    const Op& op = P.ops[i];
    HsOp& h = Q.ops[i];
    const int n_in = op.type == OP_EXT ? 0 : op.n_in;
    for (int k = 0; k < n_in; ++k) {
      const int s = src[4 * (size_t)i + k];
      h.in_off[k] = (uint16_t)off[s];
      h.in_mask[k] = (uint8_t)legs[s];
    }
    if (!is_amp_op(op.type)) {
      const int c = __builtin_popcount(legs[i]);
      const int nv = 1 << c;
      int o;
      if (!free_list[c].empty()) {
        o = free_list[c].back();
        free_list[c].pop_back();
      } else {
        const int al = nv < 4 ? nv : 4;
        top = (top + al - 1) / al * al;
        o = top;
        top += nv;
      }
      if (top > 65535) throw std::runtime_error("helicity sharing: arena beyond 65535 variants");
      off[i] = o;
      live += nv;
      if (live > Q.live_peak) Q.live_peak = live;
      h.out_off = (uint16_t)o;
      h.out_mask = (uint8_t)legs[i];
      Q.variants += nv;
      Q.lane_copies += H;
      Q.flops_event += nv * op_flop_cost(op);
      Q.flops_event_lane += (double)H * op_flop_cost(op);
      lanes_issued += (double)((nv + 31) / 32 * 32);
      if (last_read[i] < 0) {  // never read: released at once
        free_list[c].push_back(o);
        live -= nv;
      }
    } else {
      Q.amp_lanes += H;
      Q.flops_event += (double)H * op_flop_cost(op);
      Q.flops_event_lane += (double)H * op_flop_cost(op);
    }
    for (int k = 0; k < n_in; ++k) {
      const int s = src[4 * (size_t)i + k];
      bool again = false;  // the same value read twice by this op: release once
      for (int j = 0; j < k; ++j) again = again || src[4 * (size_t)i + j] == s;
      if (last_read[s] == i && !again) {
        const int c = __builtin_popcount(legs[s]);
        free_list[c].push_back(off[s]);
        live -= 1 << c;
      }
    }
  }
  Q.arena = top;
  Q.lane_use = lanes_issued > 0 ? (double)Q.variants / lanes_issued : 0.0;
  return Q;
}

std::vector<uint8_t> build_forwarding_flags(const Program& P) {
  const int n_ops = (int)P.ops.size();
  std::vector<uint8_t> fw(n_ops, 0);
  std::vector<int> holder(P.n_slots, -1), reads(n_ops, 0), last_read(n_ops, -1);
  for (int i = 0; i < n_ops; ++i) {
    const Op& op = P.ops[i];
    const int n_in = op.type == OP_EXT ? 0 : op.n_in;
    const bool prev_out = i > 0 && !is_amp_op(P.ops[i - 1].type);
    for (int k = 0; k < n_in; ++k) {
      const int src = holder.at(op.in[k]);
      if (src >= 0) {
        ++reads[src];
        last_read[src] = i;
      }
      if (prev_out && src == i - 1) fw[i] |= (uint8_t)(1u << k);
    }
    if (!is_amp_op(op.type)) holder.at(op.out) = i;
  }
  for (int i = 0; i + 1 < n_ops; ++i)
    if (!is_amp_op(P.ops[i].type) && reads[i] == 1 && last_read[i] == i + 1) fw[i] |= 16u;
  return fw;
}

HsSplitProgram build_split_shared(const Program& P, int H) {
  if (P.n_ext > 8 || P.n_ext < 5) throw std::runtime_error("split sharing: 5 to 8 legs");
  const int n_ops = (int)P.ops.size();
  const int K = P.n_ext - 3;
  std::vector<int> holder(P.n_slots, -1), last_read(n_ops, -1), reads(n_ops, 0);
  std::vector<int> src(4 * (size_t)n_ops, -1);
  std::vector<uint32_t> legs(n_ops, 0);
  for (int i = 0; i < n_ops; ++i) {
    const Op& op = P.ops[i];
    const int n_in = op.type == OP_EXT ? 0 : op.n_in;
    uint32_t u = 0;
    for (int k = 0; k < n_in; ++k) {
      const int s = holder.at(op.in[k]);
      if (s < 0) throw std::runtime_error("split sharing: slot read before it is written");
      src[4 * (size_t)i + k] = s;
      last_read[s] = i;
      ++reads[s];
      u |= legs[s];
    }
    if (!is_amp_op(op.type)) {
      legs[i] = op.type == OP_EXT ? (1u << op.leg) : u;
      holder.at(op.out) = i;
    }
  }
  HsSplitProgram Q;
  Q.levels = K;
  Q.rec.assign(n_ops, HsOp{});
  // prologue values: offsets level by level, in program order within a level
  std::vector<int> off(n_ops, -1);
  int top = 0;
  for (int lv = 1; lv <= K; ++lv) {
    for (int i = 0; i < n_ops; ++i) {
      const Op& op = P.ops[i];
      if (is_amp_op(op.type) || __builtin_popcount(legs[i]) != lv) continue;
      const int nv = 1 << lv;
      const int al = nv < 4 ? nv : 4;
      top = (top + al - 1) / al * al;
      off[i] = top;
      top += nv;
      if (top > 65535) throw std::runtime_error("split sharing: area beyond 65535 variants");
      for (int v = 0; v < nv; ++v) Q.tasks.push_back((uint32_t)i << 8 | (uint32_t)v);
      Q.prologue_variants += nv;
      Q.flops_event += nv * op_flop_cost(op);
    }
    Q.level_end.push_back((int)Q.tasks.size());
  }
  Q.area = top;
  for (int i = 0; i < n_ops; ++i) {
    const Op& op = P.ops[i];
    const bool amp = is_amp_op(op.type);
    const bool shared = !amp && __builtin_popcount(legs[i]) <= K;
    if (!amp && !shared && (reads[i] != 1 || last_read[i] != i + 1))
      throw std::runtime_error("split sharing: a longer value is not read once by the next op");
    HsOp& h = Q.rec[i];
    const int n_in = op.type == OP_EXT ? 0 : op.n_in;
    int transients = 0;
    for (int k = 0; k < n_in; ++k) {
      const int s = src[4 * (size_t)i + k];
      h.in_mask[k] = (uint8_t)legs[s];
      if (off[s] >= 0) {
        h.in_off[k] = (uint16_t)off[s];
      } else {
        h.in_off[k] = kHsTransient;
        ++transients;
        if (shared) throw std::runtime_error("split sharing: a prologue value reads a transient");
      }
    }
    if (transients > 1) throw std::runtime_error("split sharing: an op reads two transients");
    if (shared) {
      h.out_off = (uint16_t)off[i];
      h.out_mask = (uint8_t)legs[i];
    } else {
      Q.main_ops.push_back(op);
      Q.main_rec.push_back(h);
      Q.flops_event += (double)H * op_flop_cost(op);
    }
  }
  return Q;
}

}  // namespace mea
