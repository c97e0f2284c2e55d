// cg_expr.cu -- expression programs: source-transformation reverse-mode AD of
// a per-element objective term, compiled at run time for this GPU.
//
// The paper's tool differentiates C++ source by transforming it into the
// source of its reverse-mode derivative (Sec. 2-3, Listings 1-2).  Here the
// input is a small expression DAG (cg_expr_node, topological order); this
// file writes the CUDA source of
//   cgx_tiles:    per parameter point and chunk of elements (chunk-major
//                 tiles, as the hand-written kernels), the forward values
//                 and the reverse sweep of every element, summed per thread
//                 in FP64 and per block in a fixed order into partials;
//   cgx_finalize: per parameter point, the partials summed in chunk order
//                 and the reverse sweep of the parameter-only part seeded
//                 with those sums (the epilogue),
// compiles it with NVRTC (loaded with dlopen at first use) for the current
// device's architecture and loads it through the driver entry points.  The
// per-element exponentials, logarithms and divisions of cgx_tiles use the
// table-driven FP64 functions of cg_fp64.cuh (its text handed to NVRTC as an
// in-memory header; the tables are libcg's own, copied into shared memory
// from pointers passed at launch); the per-point prologue and the finalize
// keep CUDA's functions.
//
// Node classes: constant (no parameter, no element input), parameter-only
// (evaluated once per point: the prologue), input-only (per element, no
// adjoint) and mixed (per element, with adjoint).  The "frontier" is the
// set of parameter-only nodes that mixed nodes use: per element the reverse
// sweep stops there and their adjoints are accumulated; the epilogue chains
// the accumulated frontier adjoints back to the parameters once.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <dlfcn.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "cg_fp64.cuh"
#include "cg_fp64_text.inc"   // kCgFp64Text: the text of cg_fp64.cuh (written by _build.py)
#include "cg_internal.cuh"

// NVRTC entry points (resolved with dlsym; no link-time dependency)
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram* nvrtcProgram_t;
typedef nvrtcResult_t (*fn_nvrtcCreateProgram)(nvrtcProgram_t*, const char*, const char*, int, const char* const*,
                                               const char* const*);
typedef nvrtcResult_t (*fn_nvrtcCompileProgram)(nvrtcProgram_t, int, const char* const*);
typedef nvrtcResult_t (*fn_nvrtcGetSize)(nvrtcProgram_t, size_t*);
typedef nvrtcResult_t (*fn_nvrtcGetBytes)(nvrtcProgram_t, char*);
typedef nvrtcResult_t (*fn_nvrtcDestroyProgram)(nvrtcProgram_t*);

struct cg_expr_program {
    std::string source, log;
    int n_params = 0, n_inputs = 0, n_acc = 0, device = -1, value_only = 0;
    const double* t_exp2 = nullptr;   // libcg's FP64 tables on the program's device
    const double* t_log = nullptr;
    const double* t_invf = nullptr;
    CUmodule mod = nullptr;
    CUfunction f_tiles = nullptr, f_fin = nullptr;
};

namespace cg {
namespace {

struct Nvrtc {
    fn_nvrtcCreateProgram create = nullptr;
    fn_nvrtcCompileProgram compile = nullptr;
    fn_nvrtcGetSize cubin_size = nullptr, log_size = nullptr;
    fn_nvrtcGetBytes cubin = nullptr, log = nullptr;
    fn_nvrtcDestroyProgram destroy = nullptr;
    bool ok = false;
};

const Nvrtc& nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[] = {"libnvrtc.so.13", "libnvrtc.so"};
        void* h = nullptr;
        for (const char* nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return;
        n.create = (fn_nvrtcCreateProgram)dlsym(h, "nvrtcCreateProgram");
        n.compile = (fn_nvrtcCompileProgram)dlsym(h, "nvrtcCompileProgram");
        n.cubin_size = (fn_nvrtcGetSize)dlsym(h, "nvrtcGetCUBINSize");
        n.cubin = (fn_nvrtcGetBytes)dlsym(h, "nvrtcGetCUBIN");
        n.log_size = (fn_nvrtcGetSize)dlsym(h, "nvrtcGetProgramLogSize");
        n.log = (fn_nvrtcGetBytes)dlsym(h, "nvrtcGetProgramLog");
        n.destroy = (fn_nvrtcDestroyProgram)dlsym(h, "nvrtcDestroyProgram");
        n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.log_size && n.log && n.destroy;
    });
    return n;
}

struct Driver {
    PFN_cuModuleLoadData_v2000 load = nullptr;
    PFN_cuModuleGetFunction_v2000 get = nullptr;
    PFN_cuModuleUnload_v2000 unload = nullptr;
    PFN_cuLaunchKernel_v4000 launch = nullptr;
    bool ok = false;
};

const Driver& driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto get = [](const char* name, void** p) {
            cudaDriverEntryPointQueryResult q;
            return cudaGetDriverEntryPointByVersion(name, p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *p;
        };
        void *a = nullptr, *b = nullptr, *c = nullptr, *e = nullptr;
        d.ok = get("cuModuleLoadData", &a) && get("cuModuleGetFunction", &b) && get("cuModuleUnload", &c) &&
               get("cuLaunchKernel", &e);
        d.load = (PFN_cuModuleLoadData_v2000)a;
        d.get = (PFN_cuModuleGetFunction_v2000)b;
        d.unload = (PFN_cuModuleUnload_v2000)c;
        d.launch = (PFN_cuLaunchKernel_v4000)e;
    });
    return d;
}

enum Cls { K_CONST = 0, K_PARAM_ONLY = 1, K_INPUT_ONLY = 2, K_MIXED = 3 };
constexpr int kMaxExprAcc = 128;   // past about 60 the accumulators spill to local memory

struct Plan {
    std::vector<int> cls;         // per node
    std::vector<int> front;       // frontier node ids (parameter-only nodes used by mixed nodes)
    std::vector<int> front_slot;  // per node: accumulator slot (1 + frontier index) or -1
};

bool unary(int op) {
    return op == CG_EX_NEG || op == CG_EX_EXP || op == CG_EX_LOG || op == CG_EX_SQRT || op == CG_EX_ERFC ||
           op == CG_EX_POWI;
}
bool binary(int op) {
    return op == CG_EX_ADD || op == CG_EX_SUB || op == CG_EX_MUL || op == CG_EX_DIV || op == CG_EX_MAX;
}

cg_status validate_and_plan(const cg_expr_node* nd, int n, int P, int NI, Plan& pl) {
    if (!nd || n < 1 || n > CG_EXPR_MAX_NODES || P < 0 || P > CG_EXPR_MAX_PARAMS || NI < 0 ||
        NI > CG_EXPR_MAX_INPUTS)
        return CG_ERR_INVALID_ARG;
    pl.cls.assign(n, K_CONST);
    pl.front_slot.assign(n, -1);
    std::vector<int> dp(n, 0), di(n, 0);
    for (int j = 0; j < n; ++j) {
        const cg_expr_node& x = nd[j];
        switch (x.op) {
            case CG_EX_CONST:
                if (!std::isfinite(x.c)) return CG_ERR_INVALID_ARG;
                break;
            case CG_EX_PARAM:
                if (x.i < 0 || x.i >= P) return CG_ERR_INVALID_ARG;
                dp[j] = 1;
                break;
            case CG_EX_INPUT:
                if (x.i < 0 || x.i >= NI) return CG_ERR_INVALID_ARG;
                di[j] = 1;
                break;
            case CG_EX_INDEX: di[j] = 1; break;
            default:
                if (unary(x.op)) {
                    if (x.a < 0 || x.a >= j) return CG_ERR_INVALID_ARG;
                    if (x.op == CG_EX_POWI && (x.i < -16 || x.i > 16)) return CG_ERR_INVALID_ARG;
                    dp[j] = dp[x.a];
                    di[j] = di[x.a];
                } else if (binary(x.op)) {
                    if (x.a < 0 || x.a >= j || x.b < 0 || x.b >= j) return CG_ERR_INVALID_ARG;
                    dp[j] = dp[x.a] | dp[x.b];
                    di[j] = di[x.a] | di[x.b];
                } else {
                    return CG_ERR_INVALID_ARG;
                }
        }
        pl.cls[j] = dp[j] ? (di[j] ? K_MIXED : K_PARAM_ONLY) : (di[j] ? K_INPUT_ONLY : K_CONST);
    }
    const int root = n - 1;
    if (!di[root]) return CG_ERR_INVALID_ARG;   // the term must depend on the element
    for (int j = 0; j < n; ++j) {
        if (pl.cls[j] != K_MIXED) continue;
        const int ops[2] = {nd[j].a, binary(nd[j].op) ? nd[j].b : -1};
        for (int o : ops)
            if (o >= 0 && pl.cls[o] == K_PARAM_ONLY && pl.front_slot[o] < 0) {
                pl.front_slot[o] = 1 + (int)pl.front.size();
                pl.front.push_back(o);
            }
    }
    if (1 + (int)pl.front.size() > kMaxExprAcc) return CG_ERR_UNSUPPORTED;   // per-thread accumulators
    return CG_OK;
}

std::string lit(double c) {
    char b[64];
    snprintf(b, sizeof(b), "%.17g", c);
    std::string s(b);
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return "(" + s + ")";
}

std::string v(int j) { return "v" + std::to_string(j); }
std::string g(int j) { return "g" + std::to_string(j); }

std::string rv(int j) { return "r" + std::to_string(j); }

// The element's functions in cgx_tiles (fast = true): the table-driven FP64
// functions on the block's tables `tab`; CUDA's elsewhere.
std::string f_exp(const std::string& a, bool fast) { return fast ? "cg::fexp(" + a + ", tab)" : "exp(" + a + ")"; }
std::string f_log(const std::string& a, bool fast) { return fast ? "cg::flog(" + a + ", tab)" : "log(" + a + ")"; }
std::string f_div(const std::string& a, const std::string& b, bool fast) {
    return fast ? a + " * cg::frcp_any(" + b + ")" : a + " / " + b;
}

// Value of node j from the values of its operands.  recip: the divisor of a
// DIV is fixed per point and its reciprocal rv(b) is available.
std::string forward_expr(const cg_expr_node& x, bool in_tiles, bool recip = false) {
    const std::string a = x.a >= 0 ? v(x.a) : "", b = x.b >= 0 ? v(x.b) : "";
    if (x.op == CG_EX_DIV && recip) return a + " * " + rv(x.b);
    switch (x.op) {
        case CG_EX_CONST: return lit(x.c);
        case CG_EX_PARAM: return "tp[" + std::to_string(x.i) + "]";
        case CG_EX_INPUT: return in_tiles ? "__ldg(a.in" + std::to_string(x.i) + " + e)" : "0.0";
        case CG_EX_INDEX: return "(double)e";
        case CG_EX_ADD: return a + " + " + b;
        case CG_EX_SUB: return a + " - " + b;
        case CG_EX_MUL: return a + " * " + b;
        case CG_EX_DIV: return f_div(a, b, in_tiles);
        case CG_EX_NEG: return "-" + a;
        case CG_EX_EXP: return f_exp(a, in_tiles);
        case CG_EX_LOG: return f_log(a, in_tiles);
        case CG_EX_SQRT: return "sqrt(" + a + ")";
        case CG_EX_ERFC: return "erfc(" + a + ")";
        case CG_EX_POWI: {
            if (x.i == 0) return "1.0";
            std::string t = a;
            const int m = x.i < 0 ? -x.i : x.i;
            for (int k = 1; k < m; ++k) t += " * " + a;
            return x.i < 0 ? f_div("1.0", "(" + t + ")", in_tiles) : "(" + t + ")";
        }
        case CG_EX_MAX: return "(" + a + " >= " + b + " ? " + a + " : " + b + ")";
    }
    return "0.0";
}

// Adjoint contributions of node j (adjoint gj) to its operands: (operand,
// partial); fast as for forward_expr's in_tiles.
std::vector<std::pair<int, std::string>> partials(const cg_expr_node& x, int j, bool recip = false,
                                                  bool fast = false) {
    const std::string a = x.a >= 0 ? v(x.a) : "", b = x.b >= 0 ? v(x.b) : "", vj = v(j);
    std::vector<std::pair<int, std::string>> r;
    if (x.op == CG_EX_DIV && recip) return {{x.a, rv(x.b)}, {x.b, "-" + vj + " * " + rv(x.b)}};
    switch (x.op) {
        case CG_EX_ADD: r = {{x.a, "1.0"}, {x.b, "1.0"}}; break;
        case CG_EX_SUB: r = {{x.a, "1.0"}, {x.b, "-1.0"}}; break;
        case CG_EX_MUL: r = {{x.a, b}, {x.b, a}}; break;
        case CG_EX_DIV: r = {{x.a, f_div("1.0", b, fast)}, {x.b, f_div("-" + vj, b, fast)}}; break;
        case CG_EX_NEG: r = {{x.a, "-1.0"}}; break;
        case CG_EX_EXP: r = {{x.a, vj}}; break;
        case CG_EX_LOG: r = {{x.a, f_div("1.0", a, fast)}}; break;
        case CG_EX_SQRT: r = {{x.a, f_div("0.5", vj, fast)}}; break;
        case CG_EX_ERFC: r = {{x.a, "(-1.1283791670955125739 * " + f_exp("-" + a + " * " + a, fast) + ")"}}; break;
        case CG_EX_POWI: {
            if (x.i == 0) break;
            // d a^i / da = i a^(i-1)
            std::string t = "(double)" + std::to_string(x.i);
            const int m = x.i - 1;
            if (m > 0) for (int k = 0; k < m; ++k) t += " * " + a;
            else if (m < 0) {
                std::string d = a;
                for (int k = 1; k < -m; ++k) d += " * " + a;
                t = f_div(t, "(" + d + ")", fast);
            }
            r = {{x.a, "(" + t + ")"}};
            break;
        }
        case CG_EX_MAX:
            r = {{x.a, "(" + a + " >= " + b + " ? 1.0 : 0.0)"}, {x.b, "(" + a + " >= " + b + " ? 0.0 : 1.0)"}};
            break;
        default: break;
    }
    return r;
}

std::string generate(const cg_expr_node* nd, int n, int P, int NI, const Plan& pl, bool value_only) {
    const int NF = (int)pl.front.size(), NACC = value_only ? 1 : 1 + NF;
    const int root = n - 1;
    // per-element divisions by values fixed per point (constants, parameter-only
    // nodes) become products with a reciprocal taken once per point
    std::vector<char> is_recip(n, 0);
    std::vector<int> recip_po;   // parameter-only divisors (their reciprocals travel with the frontier)
    auto recip_div = [&](int j) {
        return nd[j].op == CG_EX_DIV && (pl.cls[j] == K_MIXED || pl.cls[j] == K_INPUT_ONLY) &&
               (pl.cls[nd[j].b] == K_PARAM_ONLY || pl.cls[nd[j].b] == K_CONST);
    };
    for (int j = 0; j < n; ++j)
        if (recip_div(j) && !is_recip[nd[j].b]) {
            is_recip[nd[j].b] = 1;
            if (pl.cls[nd[j].b] == K_PARAM_ONLY) recip_po.push_back(nd[j].b);
        }
    const int NR = (int)recip_po.size();
    std::string s;
    s += "// Generated by libcg (cg_expr_compile): the per-element term and its reverse-mode adjoint.\n";
    s += "#include \"cg_fp64.cuh\"\n";
    s += "typedef long long i64;\n";
    s += "#define NACC " + std::to_string(NACC) + "\n";
    s += "#define NPAR " + std::to_string(P) + "\n";
    s += "struct Args { const double* in0; const double* in1; const double* in2; const double* in3; i64 n;\n"
         "  const double* theta; int n_theta; i64 chunk; int nbx; int n_tiles; double* part;\n"
         "  const double* t_exp2; const double* t_log; const double* t_invf; };\n";
    s += "__device__ __forceinline__ double warp_sum(double x) {\n"
         "  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);\n  return x;\n}\n";
    // ---------------- tile kernel ----------------
    s += "extern \"C\" __global__ void __launch_bounds__(256) cgx_tiles(Args a) {\n";
    s += "  __shared__ double fr_s[" + std::to_string(NF + NR > 0 ? NF + NR : 1) + "];\n";
    s += "  __shared__ double red[NACC * 8];\n";
    s += "  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;\n";
    s += "  __shared__ cg::Fp64Tab tab;   // libcg's FP64 tables, copied once per block\n"
         "  for (int i = threadIdx.x; i < cg::kExp2N / 2; i += blockDim.x)\n"
         "    reinterpret_cast<double2*>(tab.exp2)[i] = __ldg(reinterpret_cast<const double2*>(a.t_exp2) + i);\n"
         "  for (int i = threadIdx.x; i < cg::kLogN; i += blockDim.x)\n"
         "    tab.logf[i] = make_double2(__ldg(a.t_log + i), __ldg(a.t_invf + i));\n"
         "  __syncthreads();\n";
    s += "  for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {\n";
    s += "    const int c = t / a.n_theta, th = t - c * a.n_theta;   // chunk-major tiles\n";
    s += "    const double* tp = a.theta + (i64)th * NPAR;\n";
    s += "    if (threadIdx.x == 0) {   // prologue: the parameter-only values the elements use\n";
    for (int j = 0; j < n; ++j)
        if (pl.cls[j] == K_PARAM_ONLY || pl.cls[j] == K_CONST)
            s += "      const double " + v(j) + " = " + forward_expr(nd[j], false) + ";\n";
    for (int f = 0; f < NF; ++f) s += "      fr_s[" + std::to_string(f) + "] = " + v(pl.front[f]) + ";\n";
    for (int r = 0; r < NR; ++r)
        s += "      fr_s[" + std::to_string(NF + r) + "] = 1.0 / " + v(recip_po[r]) + ";\n";
    s += "    }\n    __syncthreads();\n";
    for (int f = 0; f < NF; ++f)
        s += "    const double " + v(pl.front[f]) + " = fr_s[" + std::to_string(f) + "];\n";
    for (int r = 0; r < NR; ++r)
        s += "    const double " + rv(recip_po[r]) + " = fr_s[" + std::to_string(NF + r) + "];\n";
    for (int j = 0; j < n; ++j)
        if (pl.cls[j] == K_CONST) {
            s += "    const double " + v(j) + " = " + forward_expr(nd[j], false) + ";\n";
            if (is_recip[j]) s += "    const double " + rv(j) + " = 1.0 / " + v(j) + ";\n";
        }
    s += "    double acc[NACC];\n    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;\n";
    s += "    const i64 e0 = (i64)c * a.chunk;\n";
    s += "    const i64 e1 = (a.n < e0 + a.chunk) ? a.n : e0 + a.chunk;\n";
    s += "    for (i64 e = e0 + threadIdx.x; e < e1; e += blockDim.x) {\n";
    for (int j = 0; j < n; ++j)
        if (pl.cls[j] == K_INPUT_ONLY || pl.cls[j] == K_MIXED)
            s += "      const double " + v(j) + " = " + forward_expr(nd[j], true, recip_div(j)) + ";\n";
    s += "      acc[0] += " + v(root) + ";\n";
    if (pl.cls[root] == K_MIXED && !value_only) {
        // adjoints of the mixed nodes and of the frontier, reverse order
        for (int j = 0; j < n; ++j)
            if (pl.cls[j] == K_MIXED || pl.front_slot[j] >= 0)
                s += "      double " + g(j) + " = " + (j == root ? "1.0" : "0.0") + ";\n";
        for (int j = root; j >= 0; --j) {
            if (pl.cls[j] != K_MIXED) continue;
            for (auto& pr : partials(nd[j], j, recip_div(j), true)) {
                const int o = pr.first;
                if (o < 0) continue;
                if (pl.cls[o] == K_MIXED || pl.front_slot[o] >= 0)
                    s += "      " + g(o) + " += " + g(j) + " * " + pr.second + ";\n";
            }
        }
        for (int f = 0; f < NF; ++f)
            s += "      acc[" + std::to_string(1 + f) + "] += " + g(pl.front[f]) + ";\n";
    }
    s += "    }\n";
    // fixed-order block sum, partial [th][acc][chunk]
    s += "    for (int k = 0; k < NACC; ++k) {\n"
         "      const double w = warp_sum(acc[k]);\n"
         "      if (lane == 0) red[k * 8 + wid] = w;\n    }\n    __syncthreads();\n"
         "    if (threadIdx.x < NACC) {\n      double sum = 0.0;\n"
         "      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[threadIdx.x * 8 + w];\n"
         "      a.part[((i64)th * NACC + threadIdx.x) * a.nbx + c] = sum;\n    }\n    __syncthreads();\n";
    s += "  }\n}\n";
    // ---------------- finalize ----------------
    s += "extern \"C\" __global__ void cgx_finalize(const double* part, int nbx, int n_theta, const double* theta,\n"
         "                                        double* value, double* grad) {\n";
    s += "  const int th = blockIdx.x * blockDim.x + threadIdx.x;\n  if (th >= n_theta) return;\n";
    s += "  double S[NACC];\n  for (int k = 0; k < NACC; ++k) {\n    double sum = 0.0;\n"
         "    for (int cc = 0; cc < nbx; ++cc) sum += part[((i64)th * NACC + k) * nbx + cc];\n    S[k] = sum;\n  }\n";
    s += "  value[th] = S[0];\n";
    if (value_only) {
        s += "}\n";
        return s;
    }
    s += "  if (!grad) return;\n";
    s += "  const double* tp = theta + (i64)th * NPAR;\n";
    for (int j = 0; j < n; ++j)
        if (pl.cls[j] == K_PARAM_ONLY || pl.cls[j] == K_CONST)
            s += "  const double " + v(j) + " = " + forward_expr(nd[j], false) + ";\n";
    for (int j = 0; j < n; ++j)
        if (pl.cls[j] == K_PARAM_ONLY)
            s += "  double " + g(j) + " = " +
                 (pl.front_slot[j] >= 0 ? "S[" + std::to_string(pl.front_slot[j]) + "]" : std::string("0.0")) + ";\n";
    s += "  double gp[NPAR > 0 ? NPAR : 1];\n  for (int k = 0; k < NPAR; ++k) gp[k] = 0.0;\n";
    for (int j = n - 1; j >= 0; --j) {
        if (pl.cls[j] != K_PARAM_ONLY) continue;
        if (nd[j].op == CG_EX_PARAM) {
            s += "  gp[" + std::to_string(nd[j].i) + "] += " + g(j) + ";\n";
            continue;
        }
        for (auto& pr : partials(nd[j], j)) {
            const int o = pr.first;
            if (o >= 0 && pl.cls[o] == K_PARAM_ONLY) s += "  " + g(o) + " += " + g(j) + " * " + pr.second + ";\n";
        }
    }
    s += "  for (int k = 0; k < NPAR; ++k) grad[(i64)th * NPAR + k] = gp[k];\n}\n";
    (void)NI;
    return s;
}

std::string arch_option() {
    int dev = 0, maj = 0, mnr = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    return "--gpu-architecture=sm_" + std::to_string(maj * 10 + mnr) + (maj >= 9 ? "a" : "");
}

struct ExprGrid {
    int nbx, n_tiles, grid;
    int64_t chunk;
};

ExprGrid expr_grid(int64_t n, int64_t n_theta) {
    ExprGrid g;
    const int target = 4 * device_sm_count();
    int64_t nbx = (target + n_theta - 1) / n_theta;
    nbx = std::max<int64_t>(1, std::min<int64_t>(nbx, (n + 1023) / 1024));
    nbx = std::min<int64_t>(nbx, 4096);
    g.nbx = (int)nbx;
    g.chunk = (n + nbx - 1) / nbx;
    if (g.chunk < 1) g.chunk = 1;
    g.n_tiles = (int)(n_theta * nbx);
    g.grid = std::min(g.n_tiles, 4 * device_sm_count());
    return g;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

cg_status cg_expr_compile(const cg_expr_node* nodes, int n_nodes, int n_params, int n_inputs, int flags,
                          cg_expr_program** out) {
    if (!out || (flags & ~CG_EXPR_VALUE_ONLY)) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    const bool value_only = (flags & CG_EXPR_VALUE_ONLY) != 0;
    Plan pl;
    cg_status s = validate_and_plan(nodes, n_nodes, n_params, n_inputs, pl);
    if (s != CG_OK) return s;
    cg_expr_program* p = new cg_expr_program();
    p->n_params = n_params;
    p->n_inputs = n_inputs;
    p->value_only = value_only ? 1 : 0;
    p->n_acc = value_only ? 1 : 1 + (int)pl.front.size();
    p->source = generate(nodes, n_nodes, n_params, n_inputs, pl, value_only);
    const Nvrtc& nv = nvrtc();
    const Driver& dr = driver();
    if (!nv.ok || !dr.ok || cudaFree(nullptr) != cudaSuccess) {   // cudaFree(0): the runtime's context is current
        *out = p;   // source kept (cg_expr_source); not runnable
        return CG_ERR_UNSUPPORTED;
    }
    cudaGetDevice(&p->device);
    if (cudaGetSymbolAddress((void**)&p->t_exp2, g_exp2_tab) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&p->t_log, g_log_tab) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&p->t_invf, g_invf_tab) != cudaSuccess) {
        delete p;
        return CG_ERR_CUDA;
    }
    // cg_fp64.cuh as an in-memory header; its table file and the C headers it
    // names are stand-ins (the kernels read libcg's tables through pointers)
    static const char kTablesStub[] =
        "static __device__ __align__(16) const double g_exp2_tab[2] = {0.0, 0.0};\n"
        "static __device__ const double g_log_tab[1] = {0.0};\n"
        "static __device__ const double g_invf_tab[1] = {0.0};\n";
    const char* hdr_src[] = {kCgFp64Text, kTablesStub, "", ""};
    const char* hdr_name[] = {"cg_fp64.cuh", "cg_fp64_tables.inc", "math.h", "stdint.h"};
    nvrtcProgram_t prog = nullptr;
    if (nv.create(&prog, p->source.c_str(), "cg_expr.cu", 4, hdr_src, hdr_name) != 0) {
        delete p;
        return CG_ERR_CUDA;
    }
    const std::string arch = arch_option();
    const char* opts[] = {arch.c_str(), "-std=c++17"};
    const int rc = nv.compile(prog, 2, opts);
    size_t ls = 0;
    if (nv.log_size(prog, &ls) == 0 && ls > 1) {
        std::vector<char> buf(ls);
        if (nv.log(prog, buf.data()) == 0) p->log.assign(buf.data());
    }
    std::vector<char> cubin;
    size_t cs = 0;
    if (rc == 0 && nv.cubin_size(prog, &cs) == 0 && cs > 0) {
        cubin.resize(cs);
        if (nv.cubin(prog, cubin.data()) != 0) cubin.clear();
    }
    nv.destroy(&prog);
    if (cubin.empty() || dr.load(&p->mod, cubin.data()) != CUDA_SUCCESS ||
        dr.get(&p->f_tiles, p->mod, "cgx_tiles") != CUDA_SUCCESS ||
        dr.get(&p->f_fin, p->mod, "cgx_finalize") != CUDA_SUCCESS) {
        *out = p;   // kept for cg_expr_log / cg_expr_source; not runnable
        if (p->mod) dr.unload(p->mod);
        p->mod = nullptr;
        p->f_tiles = p->f_fin = nullptr;
        return CG_ERR_CUDA;
    }
    *out = p;
    return CG_OK;
}

const char* cg_expr_source(const cg_expr_program* prog) { return prog ? prog->source.c_str() : ""; }
const char* cg_expr_log(const cg_expr_program* prog) { return prog ? prog->log.c_str() : ""; }
int cg_expr_num_acc(const cg_expr_program* prog) { return prog ? prog->n_acc : -1; }

size_t cg_expr_workspace_size(const cg_expr_program* prog, int64_t n, int64_t n_theta) {
    if (!prog || n < 1 || n_theta < 1) return 0;
    const ExprGrid g = expr_grid(n, n_theta);
    return align_up((size_t)n_theta * prog->n_acc * g.nbx * sizeof(double), 256);
}

cg_status cg_expr_gradient(const cg_expr_program* prog, const double* const* inputs, int64_t n, const double* theta,
                           int64_t n_theta, double* value, double* grad, void* ws, size_t ws_bytes, void* stream) {
    if (!prog || !prog->f_tiles || n < 1 || n_theta < 1 || n_theta > (1 << 24) || !theta || !value)
        return CG_ERR_INVALID_ARG;
    if (grad && prog->value_only) return CG_ERR_INVALID_ARG;
    if (prog->n_inputs > 0 && !inputs) return CG_ERR_INVALID_ARG;
    for (int k = 0; k < prog->n_inputs; ++k)
        if (!inputs[k]) return CG_ERR_INVALID_ARG;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != prog->device) return CG_ERR_INVALID_ARG;
    if (!ws || ws_bytes < cg_expr_workspace_size(prog, n, n_theta)) return CG_ERR_WORKSPACE;
    const Driver& dr = driver();
    const ExprGrid g = expr_grid(n, n_theta);
    struct {
        const double* in[4];
        long long n;
        const double* theta;
        int n_theta;
        long long chunk;
        int nbx;
        int n_tiles;
        double* part;
        const double* t_exp2;
        const double* t_log;
        const double* t_invf;
    } args;
    memset(&args, 0, sizeof(args));
    for (int k = 0; k < prog->n_inputs; ++k) args.in[k] = inputs[k];
    args.n = n;
    args.theta = theta;
    args.n_theta = (int)n_theta;
    args.chunk = g.chunk;
    args.nbx = g.nbx;
    args.n_tiles = g.n_tiles;
    args.part = (double*)ws;
    args.t_exp2 = prog->t_exp2;
    args.t_log = prog->t_log;
    args.t_invf = prog->t_invf;
    void* p1[] = {&args};
    CUstream st = (CUstream)stream;
    prof_begin((cudaStream_t)stream);
    if (dr.launch(prog->f_tiles, (unsigned)g.grid, 1, 1, 256, 1, 1, 0, st, p1, nullptr) != CUDA_SUCCESS)
        return CG_ERR_CUDA;
    prof_end((cudaStream_t)stream);
    const double* part = (const double*)ws;
    int nbx = g.nbx, nt = (int)n_theta;
    void* p2[] = {&part, &nbx, &nt, &theta, &value, &grad};
    if (dr.launch(prog->f_fin, (unsigned)((n_theta + 127) / 128), 1, 1, 128, 1, 1, 0, st, p2, nullptr) !=
        CUDA_SUCCESS)
        return CG_ERR_CUDA;
    return CG_OK;
}

void cg_expr_free(cg_expr_program* prog) {
    if (!prog) return;
    if (prog->mod && driver().ok) driver().unload(prog->mod);
    delete prog;
}

}  // extern "C"
