// Straight-line CUDA emitter: turns a process program into a per-process
// kernel whose wavefunctions and colour amplitudes live in registers.
//
// The emitted body is the same program the interpreter runs (same ops, same
// order, same device functions from heget.cuh), written out with one SSA
// variable per op and the colour matrix as literal constants, so that nvcc
// allocates registers and schedules across ops.  It is used for the small
// processes (n_ext <= 5) whose live state fits in registers; larger processes
// stay on the table-driven interpreter.
//
// Usage (build step): mea_codegen <out.cu> <pdg,pdg,...> [<pdg,...> ...]
#include <cstdio>
#include <cstdlib>
#include <map>
#include <numeric>
#include <sstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "generator.h"

namespace {

std::string key_of(const std::vector<int>& pdg) {
  std::string k;
  for (size_t i = 0; i < pdg.size(); ++i) k += (i ? "," : "") + std::to_string(pdg[i]);
  return k;
}

std::string ident_of(const std::vector<int>& pdg) {
  std::string k = "p";
  for (int c : pdg) k += (c < 0 ? "_m" + std::to_string(-c) : "_" + std::to_string(c));
  return k;
}

std::string lit(double v) {
  char b[64];
  std::snprintf(b, sizeof b, "%.17g", v);
  std::string s(b);
  if (s.find('.') == std::string::npos && s.find('e') == std::string::npos) s += ".0";
  return "R(" + s + ")";
}

void emit_body(std::ostringstream& o, const mea::Program& P, const std::string& name) {
  using namespace mea;
  const int m = P.n_jamp;  // colour amplitudes accumulated (folded for gluons)
  o << "template <typename R>\nstruct " << name << " {\n";
  o << "  static constexpr int kColour = " << m << ";\n";
  o << "  __device__ __forceinline__ static void run(const R* __restrict__ et, const R* __restrict__ mt,\n"
       "                                             uint32_t lam, R g, R gg, double inv_den, double& val,\n"
       "                                             float& kappa) {\n";
  o << "    cx<R> J[" << m << "];\n    cx<R> Jl[" << m << "];\n";
  o << "#pragma unroll\n    for (int a = 0; a < " << m << "; ++a) { J[a] = mk<R>(R(0), R(0)); Jl[a] = J[a]; }\n";
  o << "    float mass = 0.f;\n";
  // Common factor of the colour coefficients: the amplitudes are accumulated
  // with the cofactors (+-1 for every process here) and J is scaled by the
  // factor at the end -- a power of two for the gluon processes, so the
  // result is bitwise that of accumulating the full coefficients.
  int cfac = 0;
  bool cfac_real = true;
  for (const ColEntry& c : P.col) {
    cfac = std::gcd(cfac, std::gcd(std::abs((int)c.re), std::abs((int)c.im)));
    if (c.im != 0) cfac_real = false;
  }
  if (cfac <= 0 || (cfac & (cfac - 1)) != 0) cfac = 1;  // keep the scaling exact
  std::vector<int> slot_op(P.n_slots + 1, -1);
  for (size_t i = 0; i < P.ops.size(); ++i) {
    const Op& op = P.ops[i];
    auto in = [&](int k) { return "w" + std::to_string(slot_op[op.in[k]]); };
    auto mrow = [&](int r) { return "mt + " + std::to_string(5 * r); };
    auto minv = [&](int r) { return "mt[" + std::to_string(5 * r + 4) + "]"; };
    std::string w = "w" + std::to_string(i);
    switch (op.type) {
      case OP_EXT: {
        int l = op.leg;
        std::string lam = "((lam >> " + std::to_string(l) + ") & 1u ? 1 : -1)";
        if (P.leg_type[l] == 0) {
          o << "    const W4<R> " << w << " = ext_gluon<R>(et + " << 8 * l << ", et + " << 8 * l + 3 << ", "
            << lam << ", " << (P.incoming[l] ? "false" : "true") << ");\n";
        } else {
          int kind = P.leg_type[l] == 1 ? (P.incoming[l] ? 0 : 1) : (P.incoming[l] ? 3 : 2);
          o << "    const W4<R> " << w << " = ext_spinor<R>(et[" << 8 * l << "], et[" << 8 * l + 1 << "], mk<R>(et["
            << 8 * l + 2 << "], et[" << 8 * l + 3 << "]), " << lam << ", " << kind << ");\n";
        }
        break;
      }
      case OP_JVV:
        o << "    const W4<R> " << w << " = jvv<R>(" << in(0) << ", " << in(1) << ", " << mrow(op.min[0]) << ", "
          << mrow(op.min[1]) << ", " << minv(op.mout) << ", g);\n";
        break;
      case OP_JGGG:
        o << "    const W4<R> " << w << " = jggg<R>(" << in(0) << ", " << in(1) << ", " << in(2) << ", "
          << minv(op.mout) << ", gg);\n";
        break;
      case OP_FVI:
        o << "    const W4<R> " << w << " = fvi<R>(" << in(0) << ", " << in(1) << ", " << mrow(op.mout) << ", "
          << minv(op.mout) << ", g);\n";
        break;
      case OP_FVO:
        o << "    const W4<R> " << w << " = fvo<R>(" << in(0) << ", " << in(1) << ", " << mrow(op.mout) << ", "
          << minv(op.mout) << ", g);\n";
        break;
      case OP_JIO:
        o << "    const W4<R> " << w << " = jio<R>(" << in(0) << ", " << in(1) << ", " << minv(op.mout) << ", g);\n";
        break;
      case OP_PVVV:
        o << "    const W4<R> " << w << " = vvv_part<R>(" << in(0) << ", " << in(1) << ", " << mrow(op.min[0]) << ", "
          << mrow(op.min[1]) << ", " << mrow(op.min[2]) << ", g);\n";
        break;
      case OP_PGGGG:
        o << "    const W4<R> " << w << " = gggg_part<R>(" << in(0) << ", " << in(1) << ", " << in(2) << ", gg);\n";
        break;
      case OP_PIOV:
        o << "    const W4<R> " << w << " = " << (op.leg == 0 ? "iov_part_i" : op.leg == 1 ? "iov_part_o" : "iov_part_v")
          << "<R>(" << in(0) << ", " << in(1) << ", g);\n";
        break;
      case OP_AVVV:
      case OP_AGGGG:
      case OP_AIOV:
      case OP_ADOT: {
        o << "    {\n      const cx<R> a = ";
        if (op.type == OP_ADOT)
          o << "part_contract<R>(" << in(0) << ", " << in(1) << ", " << ((op.leg & 1) ? "true" : "false") << ", "
            << ((op.leg & 2) ? "true" : "false") << ");\n";
        else if (op.type == OP_AVVV)
          o << "vvv_amp<R>(" << in(0) << ", " << in(1) << ", " << in(2) << ", " << mrow(op.min[0]) << ", "
            << mrow(op.min[1]) << ", " << mrow(op.min[2]) << ", g);\n";
        else if (op.type == OP_AGGGG)
          o << "gggg_amp<R>(" << in(0) << ", " << in(1) << ", " << in(2) << ", " << in(3) << ", gg);\n";
        else
          o << "iov_amp<R>(" << in(0) << ", " << in(1) << ", " << in(2) << ", g);\n";
        int wsum = 0;  // sum over entries of |Re c| + |Im c| (cancellation indicator)
        for (uint32_t k = 0; k < op.col_count; ++k) {
          const ColEntry& c = P.col[op.col_begin + k];
          wsum += std::abs((int)c.re) + std::abs((int)c.im);
          if (cfac_real) {
            const int n = (int)c.re / cfac;
            if (n == 1 || n == -1)
              o << "      jadd<R>(J[" << c.alpha << "], Jl[" << c.alpha << "], " << (n > 0 ? "a" : "neg<R>(a)")
                << ");\n";
            else
              o << "      jadd<R>(J[" << c.alpha << "], Jl[" << c.alpha << "], mk<R>(R(" << n << ") * a.r, R(" << n
                << ") * a.i));\n";
          } else {
            o << "      jadd<R>(J[" << c.alpha << "], Jl[" << c.alpha << "], mk<R>(R(" << (int)c.re << ") * a.r - R("
              << (int)c.im << ") * a.i, R(" << (int)c.re << ") * a.i + R(" << (int)c.im << ") * a.r));\n";
          }
        }
        o << "      if constexpr (std::is_same<R, float>::value) mass += " << wsum
          << ".f * (fabsf(a.r) + fabsf(a.i));\n";
        o << "    }\n";
        break;
      }
      default:
        throw std::runtime_error("codegen: unknown op");
    }
    if (!is_amp_op(op.type)) slot_op[op.out] = (int)i;
  }
  // colour quadratic form with the integer colour matrix (symmetric)
  o << "    cx<R> F[" << m << "];\n    float jabs = 0.f;\n";
  const std::string scale = (cfac_real && cfac != 1) ? " * R(" + std::to_string(cfac) + ")" : "";
  o << "#pragma unroll\n    for (int a = 0; a < " << m << "; ++a) { F[a] = jfin<R>(J[a], Jl[a]); F[a].r = F[a].r"
    << scale << "; F[a].i = F[a].i" << scale << "; jabs += (float)(fabs(F[a].r) + fabs(F[a].i)); }\n";
  o << "    R tot = R(0);\n";
  for (int a = 0; a < m; ++a) {
    std::ostringstream z;
    bool any = false;
    for (int b = a; b < m; ++b) {
      int64_t k = P.cf_jamp[(size_t)a * m + b];
      if (!k) continue;
      double c = (b == a) ? (double)k : 2.0 * (double)k;
      z << "      z += " << lit(c) << " * (F[" << a << "].r * F[" << b << "].r + F[" << a << "].i * F[" << b
        << "].i);\n";
      any = true;
    }
    if (any) o << "    {\n      R z = R(0);\n" << z.str() << "      tot += z;\n    }\n";
  }
  o << "    val = (double)tot * inv_den;\n";
  o << "    kappa = (jabs > 0.f) ? mass / jabs : 0.f;\n";
  o << "  }\n};\n\n";
}

}  // namespace

// Usage: mea_codegen OUT_DIR pdg,pdg,... [...]
// Writes, per process, one translation unit (device module) per kernel
// variant, OUT_DIR/generated_<process>_<variant>.cu, and
// OUT_DIR/generated_table.cu with the per-process dispatch and the table.
int main(int argc, char** argv) {
  if (argc < 3) {
    std::fprintf(stderr, "usage: %s out_dir pdg,pdg,... [...]\n", argv[0]);
    return 2;
  }
  const std::string dir = argv[1];
  auto write = [](const std::string& path, const std::string& txt) {
    FILE* f = std::fopen(path.c_str(), "w");
    if (!f) return false;
    std::fwrite(txt.data(), 1, txt.size(), f);
    std::fclose(f);
    return true;
  };
  // (suffix, real type, body, MINB, MAXT): the FP32 variants in regvar order
  // (2 * cap + body, kernels.h), then the FP64 one
  struct Variant {
    const char* suffix;
    const char* real;
    bool partials;
    int minb, maxt;
  };
  static const Variant kVariants[] = {
      {"f_part_128", "float", true, 2, 256},  {"f_diag_128", "float", false, 2, 256},
      {"f_part_85", "float", true, 3, 256},   {"f_diag_85", "float", false, 3, 256},
      {"f_part_168", "float", true, 2, 192},  {"f_diag_168", "float", false, 2, 192},
      {"d_part_128", "double", true, 2, 256}};
  const int n_f32 = 6;
  std::ostringstream t;
  t << "// Generated by mea_codegen; do not edit.\n#include \"kernels.h\"\n\nnamespace mea {\n\n";
  std::vector<std::string> ids, pdg_keys;
  for (int i = 2; i < argc; ++i) {
    std::vector<int> pdg;
    std::string s = argv[i];
    size_t pos = 0;
    while (pos < s.size()) {
      size_t e = s.find(',', pos);
      if (e == std::string::npos) e = s.size();
      pdg.push_back(std::atoi(s.substr(pos, e - pos).c_str()));
      pos = e + 1;
    }
    // two bodies per process: with vertex partials and with one vertex call
    // per diagram (fewer FLOPs against fewer live values)
    const std::string id = ident_of(pdg);
    mea::BuildOptions with, without;
    with.group_together = true;
    without.vertex_partials = false;
    std::ostringstream body_part, body_diag;
    emit_body(body_part, mea::build_program(pdg, with), "Body_" + id);
    emit_body(body_diag, mea::build_program(pdg, without), "BodyN_" + id);
    for (const Variant& v : kVariants) {
      const std::string fn = id + "_" + v.suffix;
      const std::string body = std::string(v.partials ? "Body_" : "BodyN_") + id + "<" + v.real + ">";
      const std::string targs = std::string(v.real) + ", " + body + ", " + std::to_string(v.minb) + ", " +
                                std::to_string(v.maxt);
      const std::string inst = "gen_kernel<" + targs + ">";
      std::ostringstream o;
      o << "// Generated by mea_codegen from the process generator; do not edit.\n"
           "#include \"gen_kernel.cuh\"\n\nnamespace mea {\nnamespace {\n\n"
        << (v.partials ? body_part.str() : body_diag.str()) << "}  // namespace\n\n";
      o << "void gen_launch_" << fn << "(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s) {\n"
        << "  gen_launch_v<" << targs << ">(p, c, a, s);\n}\n";
      o << "const void* gen_kernel_" << fn << "() { return reinterpret_cast<const void*>(" << inst << "); }\n\n"
        << "}  // namespace mea\n";
      if (!write(dir + "/generated_" + fn + ".cu", o.str())) return 1;
      t << "void gen_launch_" << fn << "(const DevProgram&, const AmpConfig&, const AmpLaunch&, cudaStream_t);\n"
        << "const void* gen_kernel_" << fn << "();\n";
    }
    // dispatch: regvar 0..n_f32-1 are the FP32 variants in kVariants order
    t << "static void launch_" << id << "(bool fp64, int regvar, const DevProgram& p, const AmpConfig& c, "
         "const AmpLaunch& a, cudaStream_t s) {\n"
      << "  if (fp64) return gen_launch_" << id << "_" << kVariants[n_f32].suffix << "(p, c, a, s);\n"
      << "  switch (regvar) {\n";
    for (int k = 1; k < n_f32; ++k)
      t << "    case " << k << ": return gen_launch_" << id << "_" << kVariants[k].suffix << "(p, c, a, s);\n";
    t << "    default: return gen_launch_" << id << "_" << kVariants[0].suffix << "(p, c, a, s);\n  }\n}\n";
    t << "static const void* kernel_" << id << "(bool fp64, int regvar) {\n"
      << "  if (fp64) return gen_kernel_" << id << "_" << kVariants[n_f32].suffix << "();\n"
      << "  switch (regvar) {\n";
    for (int k = 1; k < n_f32; ++k)
      t << "    case " << k << ": return gen_kernel_" << id << "_" << kVariants[k].suffix << "();\n";
    t << "    default: return gen_kernel_" << id << "_" << kVariants[0].suffix << "();\n  }\n}\n\n";
    ids.push_back(id);
    pdg_keys.push_back(key_of(pdg));
  }
  t << "const GenEntry* generated_table(int* n) {\n  static const GenEntry t[] = {\n";
  for (size_t k = 0; k < ids.size(); ++k)
    t << "    {\"" << pdg_keys[k] << "\", &launch_" << ids[k] << ", &kernel_" << ids[k] << "},\n";
  t << "  };\n  *n = " << ids.size() << ";\n  return t;\n}\n\n}  // namespace mea\n";
  if (!write(dir + "/generated_table.cu", t.str())) return 1;
  return 0;
}
