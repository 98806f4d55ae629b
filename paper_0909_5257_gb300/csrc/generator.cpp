// Process generator (host side of the CUDA path).  See generator.h.
//
// Colour bookkeeping.  Every current carries its colour as a polynomial in the
// generators of the external gluons:
//   * a gluon current without quark lines:   M = sum_w c_w T^{w_1}...T^{w_k}
//     (the matrix sum_e T^e C^e of its colour factor C^e);
//   * a gluon current that contains a complete quark line (z <- y):
//     sum_e T^e (x) (sum_w c_w  w[E -> T^e])_{z y}, stored as the line words w
//     that contain the exchanged-gluon symbol E once;
//   * a quark (antiquark) current: the string of generators met along the line;
//   * a quark current that absorbed a gluon current holding the other line:
//     pairs (line-1 word, line-2 word), each containing E once.
// The vertex colour factors are those of Sec. 4: i f^{abc} for vvvxxx/jvvxx0,
// f^{abe}f^{cde}, f^{ace}f^{dbe}, f^{ade}f^{bce} for the three ggggxx/jgggx0
// calls, -T^a for iovxx0, T^a for the qqg currents.  With
// f^{abc} T^c = -i [T^a, T^b] these become commutators of the polynomials,
// and a closing gluon leg r gives 2 Tr(T^r M).  Moving a commutator through
// the exchanged gluon uses (ad_Y)^T = -ad_Y under Tr(T^a T^b) = delta/2.
#include "generator.h"

#include <algorithm>
#include <array>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <stdexcept>
#include <unordered_map>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace mea {
namespace {

const int kNc = 3;
const int8_t kE = -1;  // exchanged-gluon symbol inside line words

// ------------------------------------------------------------ Gaussian ints
struct GI {
  int64_t re = 0, im = 0;
};
GI operator*(GI a, GI b) { return GI{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
GI operator+(GI a, GI b) { return GI{a.re + b.re, a.im + b.im}; }
bool is0(GI a) { return a.re == 0 && a.im == 0; }

typedef std::vector<int8_t> Word;
typedef std::map<Word, GI> Poly;
typedef std::map<std::pair<Word, Word>, GI> Poly2;

void acc(Poly& p, const Word& w, GI c) {
  if (is0(c)) return;
  auto it = p.find(w);
  if (it == p.end()) p.emplace(w, c);
  else {
    it->second = it->second + c;
    if (is0(it->second)) p.erase(it);
  }
}
void acc2(Poly2& p, const Word& a, const Word& b, GI c) {
  if (is0(c)) return;
  auto k = std::make_pair(a, b);
  auto it = p.find(k);
  if (it == p.end()) p.emplace(k, c);
  else {
    it->second = it->second + c;
    if (is0(it->second)) p.erase(it);
  }
}
Word cat(const Word& a, const Word& b) {
  Word r(a);
  r.insert(r.end(), b.begin(), b.end());
  return r;
}
Poly mul(const Poly& a, const Poly& b) {
  Poly r;
  for (auto& x : a)
    for (auto& y : b) acc(r, cat(x.first, y.first), x.second * y.second);
  return r;
}
Poly add(const Poly& a, const Poly& b, GI sb = GI{1, 0}) {
  Poly r = a;
  for (auto& y : b) acc(r, y.first, y.second * sb);
  return r;
}
Poly scale(const Poly& a, GI s) {
  Poly r;
  for (auto& x : a) acc(r, x.first, x.second * s);
  return r;
}
Poly comm(const Poly& a, const Poly& b) { return add(mul(a, b), mul(b, a), GI{-1, 0}); }
Poly symE() { Poly p; p[Word{kE}] = GI{1, 0}; return p; }
// Replace the single E of every word of p by the polynomial q (whose words hold E once).
Poly substE(const Poly& p, const Poly& q) {
  Poly r;
  for (auto& x : p) {
    const Word& w = x.first;
    auto it = std::find(w.begin(), w.end(), kE);
    if (it == w.end()) throw std::runtime_error("generator: word without exchanged gluon");
    Word pre(w.begin(), it), post(it + 1, w.end());
    for (auto& y : q) acc(r, cat(cat(pre, y.first), post), x.second * y.second);
  }
  return r;
}

// ------------------------------------------------------------------ legs
enum LineKind { LG = 0, LPSI = 1, LBAR = 2 };

struct Leg {
  int pdg;
  bool in;
  int kind;   // LG, LPSI (u or v wavefunction, fermion flow starts), LBAR (ubar, vbar)
  int flav;
};

// Colour object classes.
enum CClass { C_G0 = 0, C_G1 = 1, C_STR = 2, C_PAIR = 3 };

struct Node {
  int id;
  int type;              // OpType of the producing op
  int kind;              // LG, LPSI, LBAR
  int open_leg;          // LPSI: starting psi leg; LBAR: ending psibar leg; LG with a line: its psi leg
  uint32_t mask;
  std::vector<int> kids; // node ids in call order
  int cls;
  Poly p;
  Poly2 p2;
};

struct Amp {
  int type;
  std::vector<int> kids;     // node ids in call order (root leg node included)
  std::vector<std::pair<int, GI>> col;
};

struct Builder {
  std::vector<Leg> legs;
  int n = 0;
  int root = 0;
  Family fam = FAM_GLUON;
  std::vector<int> psi_legs, bar_legs;
  std::vector<std::unique_ptr<Node>> nodes;
  std::map<std::tuple<uint32_t, int, int>, std::vector<int>> memo;
  std::vector<Amp> amps;
  // basis
  std::map<Word, int> gluon_index;                                  // word (without root) -> alpha
  std::map<std::tuple<int, Word, Word>, int> pair_index;           // (psi leg of line 1, w1, w2)
  int n_colour = 0;
  std::vector<std::vector<std::pair<std::vector<int>, std::array<int, 2>>>> basis_chains;
  // per basis element: list of chains (gluon labels; label 100 = E), {row, col} (-1,-1 closed)

  int quark_count(uint32_t m, int kind, int flav) const {
    int c = 0;
    for (int l = 0; l < n; ++l)
      if ((m >> l & 1u) && legs[l].kind == kind && (flav < 0 || legs[l].flav == flav)) ++c;
    return c;
  }

  int add_node(Node nd) {
    nd.id = (int)nodes.size();
    nodes.emplace_back(new Node(std::move(nd)));
    return nodes.back()->id;
  }

  // psi leg of the complete quark line inside a gluon current mask (or -1)
  int line_psi(uint32_t m) const {
    for (int l = 0; l < n; ++l)
      if ((m >> l & 1u) && legs[l].kind == LPSI) return l;
    return -1;
  }

  const std::vector<int>& currents(uint32_t S, int kind, int leg) {
    auto key = std::make_tuple(S, kind, leg);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    std::vector<int> out;
    int pc = __builtin_popcount(S);
    if (pc == 1) {
      int l = __builtin_ctz(S);
      if (legs[l].kind == kind && (kind == LG || l == leg)) {
        Node nd;
        nd.type = OP_EXT; nd.kind = kind; nd.open_leg = (kind == LG) ? -1 : l; nd.mask = S;
        if (kind == LG) { nd.cls = C_G0; nd.p[Word{(int8_t)l}] = GI{1, 0}; }
        else { nd.cls = C_STR; nd.p[Word{}] = GI{1, 0}; }
        out.push_back(add_node(nd));
      }
    } else if (kind == LG) {
      build_gluon_currents(S, out);
    } else {
      build_quark_currents(S, kind, leg, out);
    }
    return memo.emplace(key, out).first->second;
  }

  // A gluon line from S: no quarks (class G0) or exactly one complete line (class G1).
  void build_gluon_currents(uint32_t S, std::vector<int>& out) {
    int npsi = quark_count(S, LPSI, -1), nbar = quark_count(S, LBAR, -1);
    if (npsi != nbar || npsi > 1) return;
    if (npsi == 1) {
      int y = line_psi(S), z = -1;
      for (int l = 0; l < n; ++l)
        if ((S >> l & 1u) && legs[l].kind == LBAR) z = l;
      if (legs[y].flav != legs[z].flav) return;
    }
    uint32_t low = S & (~S + 1u);
    // two blocks
    for (uint32_t A = (S - 1) & S; A; A = (A - 1) & S) {
      if (!(A & low)) continue;
      uint32_t B = S & ~A;
      // gluon x gluon (jvvxx0)
      const std::vector<int> la = currents(A, LG, -1);
      const std::vector<int> lb = currents(B, LG, -1);
      for (int a : la)
        for (int b : lb) out.push_back(make_jvv(a, b, S));
      // quark x antiquark (jioxx0): psi part in one block, psibar part in the other
      for (int swap = 0; swap < 2; ++swap) {
        uint32_t X = swap ? B : A, Y = swap ? A : B;
        int y = -1, z = -1;
        for (int l = 0; l < n; ++l) {
          if ((X >> l & 1u) && legs[l].kind == LPSI) y = l;
          if ((Y >> l & 1u) && legs[l].kind == LBAR) z = l;
        }
        if (y < 0 || z < 0) continue;
        const std::vector<int> lf = currents(X, LPSI, y);
        const std::vector<int> lo = currents(Y, LBAR, z);
        for (int f : lf)
          for (int o : lo) out.push_back(make_jio(f, o, S));
      }
    }
    // three blocks (jgggx0, three colour structures)
    for (uint32_t A = (S - 1) & S; A; A = (A - 1) & S) {
      if (!(A & low)) continue;
      uint32_t R = S & ~A;
      uint32_t lowR = R & (~R + 1u);
      for (uint32_t B = (R - 1) & R; B; B = (B - 1) & R) {
        if (!(B & lowR)) continue;
        uint32_t C = R & ~B;
        const std::vector<int> la = currents(A, LG, -1);
        const std::vector<int> lb = currents(B, LG, -1);
        const std::vector<int> lc = currents(C, LG, -1);
        for (int a : la)
          for (int b : lb)
            for (int c : lc)
              for (int v = 0; v < 3; ++v) out.push_back(make_jggg(a, b, c, v, S));
      }
    }
  }

  void build_quark_currents(uint32_t S, int kind, int leg, std::vector<int>& out) {
    if (!(S >> leg & 1u)) return;
    // fermion content: the open leg plus complete lines
    int f = legs[leg].flav;
    for (int fl = 1; fl <= 6; ++fl) {
      int d = quark_count(S, LPSI, fl) - quark_count(S, LBAR, fl);
      int want = (fl == f) ? (kind == LPSI ? 1 : -1) : 0;
      if (d != want) return;
    }
    for (uint32_t X = (S - 1) & S; X; X = (X - 1) & S) {
      if (!(X >> leg & 1u)) continue;
      uint32_t Y = S & ~X;
      const std::vector<int> lf = currents(X, kind, leg);
      const std::vector<int> lg = currents(Y, LG, -1);
      for (int a : lf)
        for (int g : lg) out.push_back(kind == LPSI ? make_fvi(a, g, S) : make_fvo(a, g, S));
    }
  }

  // ---- current constructors with their colour objects
  int make_jvv(int a, int b, uint32_t S) {
    const Node& A = *nodes[a];
    const Node& B = *nodes[b];
    Node nd;
    nd.type = OP_JVV; nd.kind = LG; nd.mask = S; nd.kids = {a, b};
    nd.open_leg = line_psi(S);
    // colour i f^{abc} -> [A, B]
    if (A.cls == C_G0 && B.cls == C_G0) { nd.cls = C_G0; nd.p = comm(A.p, B.p); }
    else if (A.cls == C_G1 && B.cls == C_G0) { nd.cls = C_G1; nd.p = substE(A.p, comm(B.p, symE())); }
    else if (A.cls == C_G0 && B.cls == C_G1) { nd.cls = C_G1; nd.p = substE(B.p, comm(symE(), A.p)); }
    else throw std::runtime_error("generator: jvv of two quark-line currents");
    return add_node(nd);
  }

  // variant v: 0 -> jgggx0(a,b,c) with f^{abe}f^{cde}: M = -[[A,B],C]
  //            1 -> jgggx0(c,a,b) with f^{ace}f^{dbe}: M = -[B,[A,C]]
  //            2 -> jgggx0(b,c,a) with f^{ade}f^{bce}: M = -[[B,C],A]
  Poly quartic_g0(int v, const Poly& A, const Poly& B, const Poly& C) {
    GI m1{-1, 0};
    if (v == 0) return scale(comm(comm(A, B), C), m1);
    if (v == 1) return scale(comm(B, comm(A, C)), m1);
    return scale(comm(comm(B, C), A), m1);
  }
  // Quartic colour with exactly one input (index `which`) holding a quark line:
  // E -> phi^T(E) with phi the map X -> M(X in slot `which`).
  Poly quartic_g1(int v, int which, const Poly& A, const Poly& B, const Poly& C) {
    Poly E = symE();
    GI m1{-1, 0};
    if (v == 0) {  // -[[A,B],C]
      if (which == 0) return scale(comm(B, comm(C, E)), m1);   // -[B,[C,E]]
      if (which == 1) return comm(A, comm(C, E));               //  [A,[C,E]]
      return comm(comm(A, B), E);                               //  [[A,B],E]
    }
    if (v == 1) {  // -[B,[A,C]]
      if (which == 0) return comm(C, comm(B, E));               //  [C,[B,E]]
      if (which == 1) return scale(comm(comm(A, C), E), m1);    // -[[A,C],E]
      return scale(comm(A, comm(B, E)), m1);                    // -[A,[B,E]]
    }
    // -[[B,C],A]
    if (which == 0) return comm(comm(B, C), E);                 //  [[B,C],E]
    if (which == 1) return scale(comm(C, comm(A, E)), m1);      // -[C,[A,E]]
    return comm(B, comm(A, E));                                 //  [B,[A,E]]
  }

  int make_jggg(int a, int b, int c, int v, uint32_t S) {
    const Node* K[3] = {nodes[a].get(), nodes[b].get(), nodes[c].get()};
    Node nd;
    nd.type = OP_JGGG; nd.kind = LG; nd.mask = S;
    nd.open_leg = line_psi(S);
    // call order of the paper's jgggx0 calls: (a,b,c), (c,a,b), (b,c,a)
    static const int order[3][3] = {{0, 1, 2}, {2, 0, 1}, {1, 2, 0}};
    int ids[3] = {a, b, c};
    for (int k = 0; k < 3; ++k) nd.kids.push_back(ids[order[v][k]]);
    int which = -1, n1 = 0;
    for (int k = 0; k < 3; ++k)
      if (K[k]->cls == C_G1) { which = k; ++n1; }
    if (n1 > 1) throw std::runtime_error("generator: jggg with two quark lines");
    if (n1 == 0) { nd.cls = C_G0; nd.p = quartic_g0(v, K[0]->p, K[1]->p, K[2]->p); }
    else {
      nd.cls = C_G1;
      Poly P[3] = {K[0]->p, K[1]->p, K[2]->p};
      Poly q = quartic_g1(v, which, P[0], P[1], P[2]);
      nd.p = substE(K[which]->p, q);
    }
    return add_node(nd);
  }

  int make_fvi(int f, int g, uint32_t S) {
    const Node& F = *nodes[f];
    const Node& G = *nodes[g];
    Node nd;
    nd.type = OP_FVI; nd.kind = LPSI; nd.mask = S; nd.kids = {f, g};
    nd.open_leg = F.open_leg;
    // colour T^a multiplies the string from the left
    if (F.cls == C_STR && G.cls == C_G0) { nd.cls = C_STR; nd.p = mul(G.p, F.p); }
    else if (F.cls == C_STR && G.cls == C_G1) {
      nd.cls = C_PAIR;
      for (auto& x : F.p)
        for (auto& y : G.p) acc2(nd.p2, cat(Word{kE}, x.first), y.first, x.second * y.second);
    } else if (F.cls == C_PAIR && G.cls == C_G0) {
      nd.cls = C_PAIR;
      for (auto& x : F.p2)
        for (auto& y : G.p) acc2(nd.p2, cat(y.first, x.first.first), x.first.second, x.second * y.second);
    } else throw std::runtime_error("generator: fvi colour");
    return add_node(nd);
  }

  int make_fvo(int o, int g, uint32_t S) {
    const Node& O = *nodes[o];
    const Node& G = *nodes[g];
    if (O.cls != C_STR || G.cls != C_G0) throw std::runtime_error("generator: fvo colour");
    Node nd;
    nd.type = OP_FVO; nd.kind = LBAR; nd.mask = S; nd.kids = {o, g};
    nd.open_leg = O.open_leg;
    nd.cls = C_STR;
    nd.p = mul(O.p, G.p);  // T^a multiplies the barred string from the right
    return add_node(nd);
  }

  int make_jio(int f, int o, uint32_t S) {
    const Node& F = *nodes[f];
    const Node& O = *nodes[o];
    if (F.cls != C_STR || O.cls != C_STR) throw std::runtime_error("generator: jio colour");
    Node nd;
    nd.type = OP_JIO; nd.kind = LG; nd.mask = S; nd.kids = {f, o};
    nd.open_leg = F.open_leg;
    nd.cls = C_G1;
    for (auto& x : O.p)
      for (auto& y : F.p) acc(nd.p, cat(cat(x.first, Word{kE}), y.first), x.second * y.second);
    return add_node(nd);
  }

  // ---- colour basis (Table 1)
  void build_basis() {
    std::vector<int> gl;
    for (int l = 0; l < n; ++l)
      if (legs[l].kind == LG && l != root) gl.push_back(l);
    if (fam == FAM_GLUON) {
      std::vector<int8_t> w(gl.begin(), gl.end());
      std::sort(w.begin(), w.end());
      do {
        gluon_index[w] = n_colour++;
        std::vector<int> labels{root};
        labels.insert(labels.end(), w.begin(), w.end());
        basis_chains.push_back({{labels, {-1, -1}}});
      } while (std::next_permutation(w.begin(), w.end()));
    } else if (fam == FAM_ONE_LINE) {
      std::vector<int8_t> w(gl.begin(), gl.end());
      std::sort(w.begin(), w.end());
      int y = psi_legs[0];
      do {
        gluon_index[w] = n_colour++;
        basis_chains.push_back({{std::vector<int>(w.begin(), w.end()), {root, y}}});
      } while (std::next_permutation(w.begin(), w.end()));
    } else {
      int ng = (int)gl.size();
      for (int y : psi_legs) {
        if (legs[y].flav != legs[root].flav) continue;
        int y2 = (y == psi_legs[0]) ? psi_legs[1] : psi_legs[0];
        int z2 = (root == bar_legs[0]) ? bar_legs[1] : bar_legs[0];
        if (legs[y2].flav != legs[z2].flav) continue;
        for (uint32_t s = 0; s < (1u << ng); ++s) {
          Word w1{kE}, w2{kE};
          for (int k = 0; k < ng; ++k) ((s >> k & 1u) ? w1 : w2).push_back((int8_t)gl[k]);
          std::sort(w1.begin(), w1.end());
          std::sort(w2.begin(), w2.end());
          Word a = w1;
          do {
            Word b = w2;
            do {
              pair_index[std::make_tuple(y, a, b)] = n_colour++;
              auto lab = [](const Word& x) {
                std::vector<int> r;
                for (int8_t c : x) r.push_back(c == kE ? 100 : (int)c);
                return r;
              };
              basis_chains.push_back({{lab(a), {root, y}}, {lab(b), {z2, y2}}});
            } while (std::next_permutation(b.begin(), b.end()));
          } while (std::next_permutation(a.begin(), a.end()));
        }
      }
    }
  }

  // ---- amplitudes and their colour coefficients
  void add_gluon_root_amp(int type, std::vector<int> kids, const Poly& M) {
    Amp a;
    a.type = type;
    a.kids = std::move(kids);
    for (auto& x : M) {  // colour 2 Tr(T^r M)
      auto it = gluon_index.find(x.first);
      if (it == gluon_index.end()) throw std::runtime_error("generator: word outside the trace basis");
      a.col.push_back({it->second, x.second * GI{2, 0}});
    }
    amps.push_back(a);
  }

  void enumerate_amplitudes() {
    uint32_t all = (1u << n) - 1u;
    uint32_t R = all & ~(1u << root);
    int rnode = currents(1u << root, legs[root].kind, legs[root].kind == LG ? -1 : root)[0];
    if (fam == FAM_GLUON) {
      uint32_t low = R & (~R + 1u);
      for (uint32_t A = (R - 1) & R; A; A = (A - 1) & R) {
        if (!(A & low)) continue;
        uint32_t B = R & ~A;
        for (int a : currents(A, LG, -1))
          for (int b : currents(B, LG, -1)) {
            // vvvxxx(a, b, r) with colour i f^{a b r} -> 2 Tr(T^r [A,B])
            add_gluon_root_amp(OP_AVVV, {a, b, rnode}, comm(nodes[a]->p, nodes[b]->p));
          }
      }
      for (uint32_t A = (R - 1) & R; A; A = (A - 1) & R) {
        if (!(A & low)) continue;
        uint32_t Rr = R & ~A;
        uint32_t lowR = Rr & (~Rr + 1u);
        for (uint32_t B = (Rr - 1) & Rr; B; B = (B - 1) & Rr) {
          if (!(B & lowR)) continue;
          uint32_t C = Rr & ~B;
          for (int a : currents(A, LG, -1))
            for (int b : currents(B, LG, -1))
              for (int c : currents(C, LG, -1))
                for (int v = 0; v < 3; ++v) {
                  // ggggxx calls (a,b,c,r), (a,c,r,b), (a,r,b,c)
                  std::vector<int> k;
                  if (v == 0) k = {a, b, c, rnode};
                  else if (v == 1) k = {a, c, rnode, b};
                  else k = {a, rnode, b, c};
                  add_gluon_root_amp(OP_AGGGG, k,
                                     quartic_g0(v, nodes[a]->p, nodes[b]->p, nodes[c]->p));
                }
        }
      }
      return;
    }
    // quark processes: the root is a psibar-type leg; iovxx0(F, root, G), colour -T^a
    for (int y : psi_legs) {
      if (legs[y].flav != legs[root].flav) continue;
      int sign = 1;
      if (fam == FAM_TWO_LINES && y != psi_legs[0]) sign = -1;  // exchanged pairing
      for (uint32_t X = R; X; X = (X - 1) & R) {
        if (!(X >> y & 1u)) continue;
        uint32_t Y = R & ~X;
        if (!Y) continue;
        for (int f : currents(X, LPSI, y))
          for (int g : currents(Y, LG, -1)) {
            const Node& F = *nodes[f];
            const Node& G = *nodes[g];
            Amp a;
            a.type = OP_AIOV;
            a.kids = {f, rnode, g};
            GI pre{-sign, 0};
            if (F.cls == C_STR && G.cls == C_G0) {
              Poly w = mul(G.p, F.p);
              for (auto& x : w) {
                auto it = gluon_index.find(x.first);
                if (it == gluon_index.end()) throw std::runtime_error("generator: word outside the string basis");
                a.col.push_back({it->second, x.second * pre});
              }
            } else if (F.cls == C_STR && G.cls == C_G1) {
              for (auto& x : F.p)
                for (auto& z : G.p) {
                  auto it = pair_index.find(std::make_tuple(y, cat(Word{kE}, x.first), z.first));
                  if (it == pair_index.end()) throw std::runtime_error("generator: pair word outside the basis");
                  a.col.push_back({it->second, x.second * z.second * pre});
                }
            } else if (F.cls == C_PAIR && G.cls == C_G0) {
              for (auto& x : F.p2)
                for (auto& z : G.p) {
                  auto it = pair_index.find(std::make_tuple(y, cat(z.first, x.first.first), x.first.second));
                  if (it == pair_index.end()) throw std::runtime_error("generator: pair word outside the basis");
                  a.col.push_back({it->second, x.second * z.second * pre});
                }
            } else {
              throw std::runtime_error("generator: amplitude colour");
            }
            // merge repeated basis entries
            std::map<int, GI> mg;
            for (auto& e : a.col) mg[e.first] = mg[e.first] + e.second;
            a.col.clear();
            for (auto& e : mg)
              if (!is0(e.second)) a.col.push_back(e);
            amps.push_back(a);
          }
      }
    }
  }
};

// ------------------------------------------------------ colour matrix
// Colour-flow evaluation of sum_c T_alpha (T_beta)^*: every generator pair is
// replaced by 1/2 (delta delta - 1/N delta delta); the closed index loops of
// each choice give N^{loops}.  Counted with a union-find over index ports.
struct UF {
  int p[160];
  void init(int n) { for (int i = 0; i < n; ++i) p[i] = i; }
  int f(int x) { while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; } return x; }
  void u(int a, int b) { a = f(a); b = f(b); if (a != b) p[a] = b; }
};

typedef std::vector<std::pair<std::vector<int>, std::array<int, 2>>> Chains;

// Returns sum over choices of (-1)^{#U1} N^{n_g - #U1 + loops} (exact integer).
int64_t colour_flow_value(const Chains& A, const Chains& B, int n_ext) {
  // collect generator occurrences: (label, chain index) in order
  struct T { int label; };
  std::vector<int> lab;                       // per T occurrence, gluon label (E of B shifted)
  std::vector<std::pair<int, int>> fixed;     // port pairs
  int ext_base = 0;
  std::vector<std::vector<int>> chains_t;
  auto add_chain = [&](const std::vector<int>& g, int row, int col, bool conj, int eoff) {
    std::vector<int> ts;
    std::vector<int> gg = g;
    if (conj) { std::reverse(gg.begin(), gg.end()); std::swap(row, col); }
    for (int x : gg) { ts.push_back((int)lab.size()); lab.push_back(x == 100 ? 100 + eoff : x); }
    chains_t.push_back(ts);
    return std::make_tuple(ts, row, col);
  };
  std::vector<std::tuple<std::vector<int>, int, int>> all;
  for (auto& c : A) all.push_back(add_chain(c.first, c.second[0], c.second[1], false, 0));
  for (auto& c : B) all.push_back(add_chain(c.first, c.second[0], c.second[1], true, 1));
  int nT = (int)lab.size();
  ext_base = 2 * nT;
  int n_nodes = ext_base + n_ext;
  if (n_nodes > 160) throw std::runtime_error("colour flow: too many ports");
  for (auto& t : all) {
    const std::vector<int>& ts = std::get<0>(t);
    int row = std::get<1>(t), col = std::get<2>(t);
    if (row < 0) {  // closed
      for (size_t k = 0; k < ts.size(); ++k)
        fixed.push_back({2 * ts[k] + 1, 2 * ts[(k + 1) % ts.size()]});
    } else if (ts.empty()) {
      fixed.push_back({ext_base + row, ext_base + col});
    } else {
      fixed.push_back({ext_base + row, 2 * ts.front()});
      for (size_t k = 0; k + 1 < ts.size(); ++k) fixed.push_back({2 * ts[k] + 1, 2 * ts[k + 1]});
      fixed.push_back({2 * ts.back() + 1, ext_base + col});
    }
  }
  // pair the generator occurrences by label
  std::map<int, std::vector<int>> occ;
  for (int i = 0; i < nT; ++i) occ[lab[i]].push_back(i);
  std::vector<std::pair<int, int>> gpairs;
  for (auto& kv : occ) {
    if (kv.second.size() != 2) throw std::runtime_error("colour flow: unpaired gluon");
    gpairs.push_back({kv.second[0], kv.second[1]});
  }
  int ng = (int)gpairs.size();
  // which external quark nodes are used (others stay isolated and must not count)
  std::vector<int> used(n_ext, 0);
  for (auto& fp : fixed) {
    if (fp.first >= ext_base) used[fp.first - ext_base] = 1;
    if (fp.second >= ext_base) used[fp.second - ext_base] = 1;
  }
  int64_t total = 0;
  UF uf;
  for (uint32_t ch = 0; ch < (1u << ng); ++ch) {
    uf.init(n_nodes);
    for (auto& fp : fixed) uf.u(fp.first, fp.second);
    int nu1 = 0;
    for (int k = 0; k < ng; ++k) {
      int i = gpairs[k].first, j = gpairs[k].second;
      if (ch >> k & 1u) {  // -1/N delta_ij delta_kl: each generator closes on itself
        uf.u(2 * i, 2 * i + 1);
        uf.u(2 * j, 2 * j + 1);
        ++nu1;
      } else {             // delta_il delta_kj
        uf.u(2 * i, 2 * j + 1);
        uf.u(2 * j, 2 * i + 1);
      }
    }
    int loops = 0;
    for (int x = 0; x < n_nodes; ++x) {
      if (x >= ext_base && !used[x - ext_base]) continue;
      if (uf.f(x) == x) ++loops;
    }
    int64_t v = 1;
    for (int k = 0; k < ng - nu1 + loops; ++k) v *= kNc;
    total += (nu1 & 1) ? -v : v;
  }
  return total;
}

int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}

// Gluon traces: N_{sigma,tau} depends only on tau relabelled by sigma^{-1}.
void colour_matrix(Builder& B, Program& P) {
  int m = B.n_colour;
  P.cf_num.assign((size_t)m * m, 0);
  int ng_labels = 0;
  for (auto& c : B.basis_chains[0])
    for (int x : c.first) ng_labels += (x < 100) ? 1 : 0;
  // number of generator pairs: gluon labels + internal exchanged gluons (two lines: 2)
  int n_pairs = ng_labels + (B.fam == FAM_TWO_LINES ? 2 : 0);
  int64_t den = (int64_t)P.n_a * P.n_b;
  for (int k = 0; k < n_pairs; ++k) den *= 2 * kNc;
  if (B.fam == FAM_GLUON) {
    // position-relabelled cache
    std::map<std::vector<int>, int64_t> cache;
    std::vector<std::vector<int>> words(m);
    for (int a = 0; a < m; ++a) words[a] = B.basis_chains[a][0].first;
    // relabel tau by sigma's positions, then rotate to start at label 0
    std::vector<std::vector<int>> keys((size_t)m * m);
    std::set<std::vector<int>> need;
    for (int a = 0; a < m; ++a) {
      std::vector<int> pos(64, -1);
      for (size_t k = 0; k < words[a].size(); ++k) pos[words[a][k]] = (int)k;
      for (int b = a; b < m; ++b) {
        std::vector<int> t;
        for (int x : words[b]) t.push_back(pos[x]);
        auto it = std::min_element(t.begin(), t.end());
        std::rotate(t.begin(), it, t.end());
        keys[(size_t)a * m + b] = t;
        need.insert(t);
      }
    }
    std::vector<std::vector<int>> todo(need.begin(), need.end());
    std::vector<int64_t> vals(todo.size());
    std::vector<int> ident(words[0].size());
    std::iota(ident.begin(), ident.end(), 0);
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < (long)todo.size(); ++i) {
      Chains a{{ident, {-1, -1}}}, b{{todo[i], {-1, -1}}};
      vals[i] = colour_flow_value(a, b, 0);
    }
    for (size_t i = 0; i < todo.size(); ++i) cache[todo[i]] = vals[i];
    for (int a = 0; a < m; ++a)
      for (int b = a; b < m; ++b) {
        int64_t v = cache[keys[(size_t)a * m + b]];
        P.cf_num[(size_t)a * m + b] = v;
        P.cf_num[(size_t)b * m + a] = v;
      }
  } else {
#pragma omp parallel for schedule(dynamic, 8)
    for (long a = 0; a < m; ++a)
      for (int b = (int)a; b < m; ++b) {
        int64_t v = colour_flow_value(B.basis_chains[a], B.basis_chains[b], B.n);
        P.cf_num[(size_t)a * m + b] = v;
        P.cf_num[(size_t)b * m + a] = v;
      }
  }
  int64_t g = den;
  for (int64_t v : P.cf_num) g = gcd64(g, v);
  if (g == 0) g = 1;
  P.cf_den = den / g;
  P.cf_max_abs = 0;
  for (int64_t& v : P.cf_num) {
    v /= g;
    P.cf_max_abs = std::max<int64_t>(P.cf_max_abs, v < 0 ? -v : v);
  }
}

// ------------------------------------------------------ reflection folding
// Pure-gluon colour amplitudes obey J_rev(a) = (-1)^n J_a (reversing a trace
// Tr(T^r T^w1 ... T^wk) gives Tr(T^r T^wk ... T^w1) and every f^{abc} changes
// sign under the reversal of its trace expansion).  When every diagram's
// coefficients satisfy it exactly, keep the canonical half of the orderings
// (word < reversed word) and fold the colour matrix.
void fold_reflection(Builder& B, Program& P) {
  const int m = B.n_colour;
  P.n_jamp = m;
  P.cf_jamp = P.cf_num;
  if (B.fam != FAM_GLUON || m < 2) {
    P.cf_jamp_max_abs = P.cf_max_abs;
    return;
  }
  std::vector<int> rev(m, -1);
  for (auto& kv : B.gluon_index) {
    Word r = kv.first;
    std::reverse(r.begin(), r.end());
    rev[kv.second] = B.gluon_index.at(r);
  }
  const int sgn = (B.n % 2 == 0) ? 1 : -1;
  for (const Op& op : P.ops) {
    if (!is_amp_op(op.type)) continue;
    std::map<int, std::pair<int, int>> c;
    for (uint32_t k = 0; k < op.col_count; ++k) {
      const ColEntry& e = P.col[op.col_begin + k];
      c[e.alpha] = {e.re, e.im};
    }
    for (auto& kv : c) {
      auto it = c.find(rev[kv.first]);
      if (it == c.end() || it->second.first != sgn * kv.second.first || it->second.second != sgn * kv.second.second) {
        P.cf_jamp_max_abs = P.cf_max_abs;
        return;  // identity does not hold term by term: keep the full basis
      }
    }
  }
  // canonical = word lexicographically smaller than its reverse
  std::vector<int> canon_of(m, -1);
  std::vector<int> canon;
  for (auto& kv : B.gluon_index) {
    Word r = kv.first;
    std::reverse(r.begin(), r.end());
    if (kv.first < r) {
      canon_of[kv.second] = (int)canon.size();
      canon.push_back(kv.second);
    }
  }
  const int h = (int)canon.size();
  // remap colour entries, dropping the reflected ones
  std::vector<ColEntry> col;
  for (Op& op : P.ops) {
    if (!is_amp_op(op.type)) continue;
    uint32_t b = (uint32_t)col.size();
    for (uint32_t k = 0; k < op.col_count; ++k) {
      ColEntry e = P.col[op.col_begin + k];
      if (canon_of[e.alpha] < 0) continue;
      e.alpha = (uint16_t)canon_of[e.alpha];
      col.push_back(e);
    }
    op.col_begin = b;
    op.col_count = (uint32_t)col.size() - b;
  }
  P.col = col;
  P.n_jamp = h;
  P.cf_jamp.assign((size_t)h * h, 0);
  P.cf_jamp_max_abs = 0;
  for (int a = 0; a < h; ++a)
    for (int b = 0; b < h; ++b) {
      int ia = canon[a], ib = canon[b];
      int64_t v = 2 * (P.cf_num[(size_t)ia * m + ib] + sgn * P.cf_num[(size_t)ia * m + rev[ib]]);
      P.cf_jamp[(size_t)a * h + b] = v;
      P.cf_jamp_max_abs = std::max<int64_t>(P.cf_jamp_max_abs, v < 0 ? -v : v);
    }
}

// ------------------------------------------------------ helicity rules
// Massless tree amplitudes: helicity is conserved along every quark line
// (in the all-outgoing convention its two ends have opposite helicity); pure
// gluon amplitudes need at least two gluons of each helicity; with one quark
// line the gluons may not all share one helicity.
bool helicity_allowed(const Builder& B, const std::vector<int>& lam) {
  int n = B.n;
  std::vector<int> h(n);
  for (int l = 0; l < n; ++l) h[l] = B.legs[l].in ? -lam[l] : lam[l];
  if (B.fam == FAM_GLUON) {
    int np = 0;
    for (int l = 0; l < n; ++l) np += h[l] > 0;
    return np >= 2 && np <= n - 2;
  }
  if (B.fam == FAM_ONE_LINE) {
    int y = B.psi_legs[0], z = B.bar_legs[0];
    if (h[y] != -h[z]) return false;
    int np = 0, ng = 0;
    for (int l = 0; l < n; ++l)
      if (B.legs[l].kind == LG) { ++ng; np += h[l] > 0; }
    return np > 0 && np < ng;
  }
  // two lines: some flavour-consistent pairing conserves helicity on both lines
  for (int k = 0; k < 2; ++k) {
    int y1 = B.psi_legs[k], y2 = B.psi_legs[1 - k];
    int z1 = B.bar_legs[0], z2 = B.bar_legs[1];
    if (B.legs[y1].flav != B.legs[z1].flav || B.legs[y2].flav != B.legs[z2].flav) continue;
    if (h[y1] == -h[z1] && h[y2] == -h[z2]) return true;
  }
  return false;
}

// Algorithmic real-FLOP cost of each operation, counted from heget.cuh with
// real add/sub/mul = 1, complex mul = 6, complex add = 2, real x complex = 2:
// complex 4-vector dot = 30, real.complex dot = 14, slash(V) psi = 64,
// slash(P) psi = 42.  Vertex partials: the ops that make them, and one
// contraction (30) per diagram.
double op_flops(int type) {
  switch (type) {
    case OP_EXT: return 12;
    case OP_JVV: return 160;  // the ggg partial (148), the open momentum and 1/q^2
    case OP_JGGG: return 128;  // the gggg partial (120) and 1/q^2
    case OP_FVI: return 115;
    case OP_FVO: return 115;
    case OP_JIO: return 129;
    case OP_AVVV: return 178;  // the ggg partial closed with the third wavefunction
    case OP_AGGGG: return 150;  // the gggg partial closed with the fourth
    case OP_AIOV: return 96;
    case OP_ADOT: return 30;
    case OP_PVVV: return 148;
    case OP_PGGGG: return 120;
    case OP_PIOV: return 72;  // fo slash(V) or slash(V) fi, scaled (the vector fo gamma fi: 128)
  }
  return 0;
}
double op_cost(const Op& op) { return (op.type == OP_PIOV && op.leg == 2) ? 128 : op_flops(op.type); }

}  // namespace

double op_flop_cost(const Op& op) { return op_cost(op); }

Program build_program(const std::vector<int>& pdg, const BuildOptions& opt) {
  Program P;
  Builder B;
  int n = (int)pdg.size();
  if (n < 4 || n > 7) throw std::runtime_error("n_ext must be between 4 and 7");
  B.n = n;
  P.n_ext = n;
  P.pdg = pdg;
  for (int l = 0; l < n; ++l) {
    Leg g;
    g.pdg = pdg[l];
    g.in = l < 2;
    int c = pdg[l];
    if (c == 21) { g.kind = LG; g.flav = 0; }
    else if (c >= 1 && c <= 5) { g.kind = g.in ? LPSI : LBAR; g.flav = c; }
    else if (c <= -1 && c >= -5) { g.kind = g.in ? LBAR : LPSI; g.flav = -c; }
    else throw std::runtime_error("unsupported parton code " + std::to_string(c));
    B.legs.push_back(g);
    if (g.kind == LPSI) B.psi_legs.push_back(l);
    if (g.kind == LBAR) B.bar_legs.push_back(l);
    P.incoming.push_back(g.in ? 1 : 0);
    P.leg_type.push_back(g.kind);
    P.leg_is_quark.push_back(c > 0 && c != 21 ? 1 : 0);
  }
  if (B.psi_legs.size() != B.bar_legs.size()) throw std::runtime_error("quark number not conserved");
  if (B.psi_legs.empty()) { B.fam = FAM_GLUON; B.root = n - 1; }
  else if (B.psi_legs.size() == 1) { B.fam = FAM_ONE_LINE; B.root = B.bar_legs[0]; }
  else if (B.psi_legs.size() == 2) { B.fam = FAM_TWO_LINES; B.root = B.bar_legs[0]; }
  else throw std::runtime_error("more than two quark lines are not supported");
  if (B.fam == FAM_ONE_LINE && B.legs[B.psi_legs[0]].flav != B.legs[B.bar_legs[0]].flav)
    throw std::runtime_error("flavour not conserved");
  P.family = B.fam;
  P.root = B.root;
  P.n_a = pdg[0] == 21 ? 8 : 3;
  P.n_b = pdg[1] == 21 ? 8 : 3;

  B.build_basis();
  B.enumerate_amplitudes();
  if (B.amps.empty()) throw std::runtime_error("process has no tree diagrams");
  P.n_diagrams = (int)B.amps.size();
  P.n_colour = B.n_colour;

  // ---- vertex partials.  Every amplitude vertex is linear in each input; an
  // amplitude whose vertex shares all inputs but one with other amplitudes
  // joins their group, which computes the partial vertex once (one op) and
  // contracts it with each member's free input (one op per diagram).  Each
  // amplitude takes, among its possible free inputs, the one whose shared
  // remainder occurs most often; groups of one stay plain vertex calls.
  struct Choice {
    std::vector<int> key;   // {partial op, shared node ids..., free-input mask}
    int free_k = -1;        // index of the free input in the amplitude's kids
    bool neg = false;       // contraction negated (ggggxx orientation)
  };
  auto candidates = [&](const Amp& a) {
    std::vector<Choice> out;
    const std::vector<int>& x = a.kids;
    if (a.type == OP_AVVV) {
      for (int k = 0; k < 3; ++k) {  // cyclic shift: free x[k], shared (x[k+1], x[k+2])
        int b = x[(k + 1) % 3], c = x[(k + 2) % 3];
        out.push_back({{OP_PVVV, b, c, (int)B.nodes[x[k]]->mask}, k, false});
      }
    } else if (a.type == OP_AGGGG) {
      // ggggxx(a,b,c,d) = a.G(b,c,d) = b.G(a,d,c) = c.G(d,a,b) = d.G(c,b,a), G(x,y,z) = -G(x,z,y)
      static const int arg[4][3] = {{1, 2, 3}, {0, 3, 2}, {3, 0, 1}, {2, 1, 0}};
      for (int k = 0; k < 4; ++k) {
        int gx = x[arg[k][0]], gy = x[arg[k][1]], gz = x[arg[k][2]];
        out.push_back({{OP_PGGGG, gx, std::min(gy, gz), std::max(gy, gz)}, k, gy > gz});
      }
    } else if (a.type == OP_AIOV) {  // kids (fi, fo, V)
      out.push_back({{OP_PIOV, 0, x[1], x[2]}, 0, false});
      out.push_back({{OP_PIOV, 1, x[0], x[2]}, 1, false});
      out.push_back({{OP_PIOV, 2, x[0], x[1]}, 2, false});
    }
    return out;
  };
  const int n_amp = (int)B.amps.size();
  std::vector<Choice> choice(n_amp);
  {
    std::map<std::vector<int>, int> freq;
    std::vector<std::vector<Choice>> cand(n_amp);
    for (int i = 0; i < n_amp && opt.vertex_partials; ++i) {
      cand[i] = candidates(B.amps[i]);
      for (auto& c : cand[i]) freq[c.key]++;
    }
    std::map<std::vector<int>, int> taken;
    for (int i = 0; i < n_amp; ++i) {
      if (cand[i].empty()) continue;
      size_t best = 0;
      for (size_t k = 1; k < cand[i].size(); ++k)
        if (freq[cand[i][k].key] > freq[cand[i][best].key]) best = k;
      choice[i] = cand[i][best];
      taken[choice[i].key]++;
    }
    for (int i = 0; i < n_amp; ++i)
      if (choice[i].free_k >= 0 && taken[choice[i].key] < 2) choice[i] = Choice();
  }
  // groups: amplitudes sharing one partial (the shared inputs in the partial's call order)
  struct Group {
    std::vector<int> shared;
    std::vector<int> members;
  };
  std::vector<Group> groups;
  std::vector<int> group_of(n_amp, -1);
  {
    std::map<std::vector<int>, int> gid;
    for (int i = 0; i < n_amp; ++i) {
      if (choice[i].free_k < 0) continue;
      const Amp& a = B.amps[i];
      auto it = gid.find(choice[i].key);
      if (it == gid.end()) {
        Group gr;
        const int k = choice[i].free_k;
        if (a.type == OP_AVVV) gr.shared = {a.kids[(k + 1) % 3], a.kids[(k + 2) % 3]};
        else if (a.type == OP_AGGGG) gr.shared = {choice[i].key[1], choice[i].key[2], choice[i].key[3]};
        else
          for (int j = 0; j < 3; ++j)
            if (j != k) gr.shared.push_back(a.kids[j]);
        it = gid.emplace(choice[i].key, (int)groups.size()).first;
        groups.push_back(gr);
      }
      group_of[i] = it->second;
      groups[it->second].members.push_back(i);
    }
  }
  const int n_groups = (int)groups.size();

  // ---- schedule: amplitudes in a given order, currents on demand, a group's
  // partial made before its first member, every slot freed after its last use.
  // Two orders: amplitudes sorted by their largest input current, and groups
  // kept together (sorted by their shared inputs, members by their free
  // input).  The one with fewer live slots is kept unless the options ask for
  // groups together.
  const int nn = (int)B.nodes.size();
  std::vector<char> needed(nn, 0);
  std::function<void(int)> mark = [&](int id) {
    if (needed[id]) return;
    needed[id] = 1;
    for (int k : B.nodes[id]->kids) mark(k);
  };
  for (auto& a : B.amps)
    for (int k : a.kids) mark(k);
  std::vector<int> uses0(nn + n_groups, 0);  // value ids: nodes, then one partial per group
  for (int id = 0; id < nn; ++id)
    if (needed[id])
      for (int k : B.nodes[id]->kids) uses0[k]++;
  for (int i = 0; i < n_amp; ++i)
    if (group_of[i] < 0)
      for (int k : B.amps[i].kids) uses0[k]++;
    else
      uses0[B.amps[i].kids[choice[i].free_k]]++;
  for (int gI = 0; gI < n_groups; ++gI) {
    for (int k : groups[gI].shared) uses0[k]++;
    uses0[nn + gI] = (int)groups[gI].members.size();
  }
  auto sorted_desc = [](std::vector<int> k) {
    std::sort(k.rbegin(), k.rend());
    return k;
  };
  std::vector<std::vector<int>> orders;
  {
    std::vector<int> o(n_amp);
    std::iota(o.begin(), o.end(), 0);
    std::vector<std::vector<int>> key(n_amp);
    for (int i = 0; i < n_amp; ++i) key[i] = sorted_desc(B.amps[i].kids);
    std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return key[a] < key[b]; });
    orders.push_back(o);
    // groups together
    std::vector<std::pair<std::vector<int>, std::vector<int>>> units;  // (sort key, amplitudes)
    for (int i : o)
      if (group_of[i] < 0) units.push_back({key[i], {i}});
    for (const Group& gr : groups) {
      std::vector<int> m = gr.members;
      std::stable_sort(m.begin(), m.end(), [&](int a, int b) {
        return B.amps[a].kids[choice[a].free_k] > B.amps[b].kids[choice[b].free_k];
      });
      units.push_back({sorted_desc(gr.shared), m});
    }
    std::stable_sort(units.begin(), units.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    std::vector<int> o2;
    for (auto& u : units) o2.insert(o2.end(), u.second.begin(), u.second.end());
    orders.push_back(o2);
  }

  std::map<uint32_t, int> mask_row;
  auto row_of = [&](uint32_t m) {
    auto it = mask_row.find(m);
    if (it != mask_row.end()) return it->second;
    int r = (int)P.masks.size();
    P.masks.push_back(m);
    mask_row[m] = r;
    return r;
  };
  double flops = 0;
  int n_cur = 0, n_part = 0, n_slots = 0;
  std::vector<int> vertex_type;  // vertex function of each emitted amplitude op, in program order
  // Runs the schedule of `order`; emits the ops when emit is set.  Returns the slot count.
  auto run = [&](const std::vector<int>& order, bool emit) {
    std::vector<int> uses = uses0;
    std::vector<int> slot(nn + n_groups, -1);
    std::vector<int> free_slots;
    int ns = 0;
    auto alloc = [&]() {
      if (!free_slots.empty()) { int s = free_slots.back(); free_slots.pop_back(); return s; }
      return ns++;
    };
    auto release = [&](int id) {
      if (--uses[id] == 0) free_slots.push_back(slot[id]);
    };
    std::function<void(int)> ensure = [&](int id) {
      if (slot[id] >= 0) return;
      Node& nd = *B.nodes[id];
      for (int k : nd.kids) ensure(k);
      Op op;
      std::memset(&op, 0, sizeof(op));
      if (emit) {
        op.type = (uint8_t)nd.type;
        op.n_in = (uint8_t)nd.kids.size();
        for (size_t k = 0; k < nd.kids.size(); ++k) {
          op.in[k] = (uint16_t)slot[nd.kids[k]];
          op.min[k] = (uint16_t)row_of(B.nodes[nd.kids[k]]->mask);
        }
        op.mout = (uint16_t)row_of(nd.mask);
        if (nd.type == OP_EXT) op.leg = (uint16_t)__builtin_ctz(nd.mask);
      }
      for (int k : nd.kids) release(k);
      slot[id] = alloc();
      if (emit) {
        op.out = (uint16_t)slot[id];
        P.ops.push_back(op);
        flops += op_flops(nd.type);
        if (nd.type != OP_EXT) ++n_cur;
      }
    };
    auto add_colour = [&](Op& op, const Amp& a) {
      op.col_begin = (uint32_t)P.col.size();
      for (auto& e : a.col) {
        if (e.second.re < -127 || e.second.re > 127 || e.second.im < -127 || e.second.im > 127)
          throw std::runtime_error("generator: colour coefficient out of int8 range");
        P.col.push_back(ColEntry{(uint16_t)e.first, (int8_t)e.second.re, (int8_t)e.second.im});
      }
      op.col_count = (uint32_t)a.col.size();
    };
    for (int i : order) {
      const Amp& a = B.amps[i];
      const int gI = group_of[i];
      if (gI < 0) {  // plain vertex amplitude
        for (int k : a.kids) ensure(k);
        if (emit) {
          Op op;
          std::memset(&op, 0, sizeof(op));
          op.type = (uint8_t)a.type;
          op.n_in = (uint8_t)a.kids.size();
          for (size_t k = 0; k < a.kids.size(); ++k) {
            op.in[k] = (uint16_t)slot[a.kids[k]];
            op.min[k] = (uint16_t)row_of(B.nodes[a.kids[k]]->mask);
          }
          add_colour(op, a);
          P.ops.push_back(op);
          vertex_type.push_back(a.type);
          flops += op_flops(a.type) + 4.0 * a.col.size();
        }
        for (int k : a.kids) release(k);
        continue;
      }
      const Group& gr = groups[gI];
      if (slot[nn + gI] < 0) {  // the group's partial, before its first member
        const Amp& a0 = B.amps[gr.members[0]];
        const Choice& c0 = choice[gr.members[0]];
        for (int k : gr.shared) ensure(k);
        Op pop;
        std::memset(&pop, 0, sizeof(pop));
        if (emit) {
          pop.type = (uint8_t)c0.key[0];
          pop.n_in = (uint8_t)gr.shared.size();
          for (size_t k = 0; k < gr.shared.size(); ++k) {
            pop.in[k] = (uint16_t)slot[gr.shared[k]];
            pop.min[k + (a0.type == OP_AVVV ? 1 : 0)] = (uint16_t)row_of(B.nodes[gr.shared[k]]->mask);
          }
          if (a0.type == OP_AVVV) pop.min[0] = (uint16_t)row_of(B.nodes[a0.kids[c0.free_k]]->mask);
          if (a0.type == OP_AIOV) pop.leg = (uint16_t)c0.free_k;
        }
        for (int k : gr.shared) release(k);
        slot[nn + gI] = alloc();
        if (emit) {
          pop.out = (uint16_t)slot[nn + gI];
          P.ops.push_back(pop);
          flops += op_cost(pop);
          ++n_part;
        }
      }
      const int fr = a.kids[choice[i].free_k];
      ensure(fr);
      if (emit) {
        Op op;
        std::memset(&op, 0, sizeof(op));
        op.type = OP_ADOT;
        op.n_in = 2;
        op.in[0] = (uint16_t)slot[fr];
        op.in[1] = (uint16_t)slot[nn + gI];
        op.min[0] = (uint16_t)row_of(B.nodes[fr]->mask);
        const bool plain = a.type == OP_AIOV && choice[i].free_k != 2;
        op.leg = (uint16_t)((plain ? 1 : 0) | (choice[i].neg ? 2 : 0));
        add_colour(op, a);
        P.ops.push_back(op);
        vertex_type.push_back(a.type);
        flops += op_flops(OP_ADOT) + 4.0 * a.col.size();
      }
      release(fr);
      release(nn + gI);
    }
    return ns;
  };
  size_t best = 0;
  if (opt.group_together && n_groups > 0) {
    best = 1;
  } else {
    int best_slots = run(orders[0], false);
    for (size_t k = 1; k < orders.size(); ++k) {
      const int ns = run(orders[k], false);
      if (ns < best_slots) { best_slots = ns; best = k; }
    }
  }
  n_slots = run(orders[best], true);
  // Canonical mask-table numbering, so that programs built with different
  // options -- the straight-line kernels' bodies and the runtime program whose
  // table the kernels read -- agree on every row: the order in which the
  // schedule without vertex partials (amplitudes by their largest input
  // current, currents on demand) first uses each mask.  Every row field of
  // every op is remapped (unused fields are never read).
  {
    std::vector<uint32_t> canon;
    std::map<uint32_t, int> rank;
    auto use = [&](uint32_t m) {
      if (rank.emplace(m, (int)canon.size()).second) canon.push_back(m);
    };
    std::vector<char> done(nn, 0);
    std::function<void(int)> visit = [&](int id) {
      if (done[id]) return;
      done[id] = 1;
      const Node& nd = *B.nodes[id];
      for (int k : nd.kids) visit(k);
      for (int k : nd.kids) use(B.nodes[k]->mask);
      use(nd.mask);
    };
    for (int i : orders[0]) {
      for (int k : B.amps[i].kids) visit(k);
      for (int k : B.amps[i].kids) use(B.nodes[k]->mask);
    }
    if (canon.size() != P.masks.size()) throw std::runtime_error("generator: mask table mismatch");
    std::vector<uint16_t> remap(P.masks.size());
    for (size_t r = 0; r < P.masks.size(); ++r) {
      auto it = rank.find(P.masks[r]);
      if (it == rank.end()) throw std::runtime_error("generator: mask outside the canonical table");
      remap[r] = (uint16_t)it->second;
    }
    for (Op& op : P.ops) {
      for (int k = 0; k < 4; ++k) op.min[k] = remap[op.min[k]];
      op.mout = remap[op.mout];
    }
    P.masks = canon;
  }
  if (n_slots > 65535 || P.masks.size() > 65535 || B.n_colour > 65535)
    throw std::runtime_error("generator: program too large");
  P.n_slots = n_slots;
  P.n_currents = n_cur;
  P.n_partials = n_part;
  P.flops_per_hel = flops;  // recounted after the colour folding below

  colour_matrix(B, P);
  fold_reflection(B, P);
  // amplitude ops carry their diagram ordinal (program order) in `out`
  {
    uint16_t d = 0;
    for (Op& op : P.ops)
      if (is_amp_op(op.type)) op.out = d++;
  }
  {
    double f = 0, fp = 0;
    size_t k = 0;
    for (const Op& op : P.ops) {
      const double col = is_amp_op(op.type) ? 4.0 * op.col_count : 0.0;
      f += op_cost(op) + col;
      if (is_amp_op(op.type)) fp += op_flops(vertex_type[k++]) + col;
      else if (!is_partial_op(op.type)) fp += op_cost(op);
    }
    P.flops_per_hel = f;
    P.flops_per_hel_plain = fp;
  }

  // helicities
  for (int h = 0; h < (1 << n); ++h) {
    std::vector<int> lam(n);
    for (int l = 0; l < n; ++l) lam[l] = (h >> (n - 1 - l) & 1) ? 1 : -1;
    for (int l = 0; l < n; ++l) P.hel_all.push_back((int8_t)lam[l]);
    if (helicity_allowed(B, lam)) {
      for (int l = 0; l < n; ++l) P.hel.push_back((int8_t)lam[l]);
      P.n_hel++;
    }
  }
  return P;
}

int count_unique_colour_values(const Program& p) {
  std::set<int64_t> v;
  int m = p.n_colour;
  for (int a = 0; a < m; ++a)
    for (int b = a; b < m; ++b)
      if (p.cf_num[(size_t)a * m + b] != 0) v.insert(p.cf_num[(size_t)a * m + b]);
  return (int)v.size();
}

}  // namespace mea
