// Decoders specialised to one polar code ("unrolled decoder", Sec. III-B of
// Giard et al., arXiv 1504.00353): the depth-first Fast-SSC operation list of
// the code (Listing 1 is this list for the (8,5) code) is written out as CUDA
// source in which every node size and offset is a compile-time constant, then
// compiled at run time with NVRTC for the current GPU and loaded with
// cudaLibraryLoadData.
//
// Compared with the operation-list interpreter this removes, per operation,
// the decode of the op word and the indirect branch to its handler (on one warp
// these cost several times the operation itself), folds every address and loop
// bound, and lets subtrees of up to reg_subtree leaves run entirely in
// registers with statically indexed stages (see polar::RegSub in polar_ops.cuh).
// Memory-resident operations call the same device functions as the
// interpreter, with constant arguments.
#include <dlfcn.h>

#include <algorithm>
#include <map>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <cuda.h>
#include <nvrtc.h>

#include "polar_internal.h"

namespace polar {
namespace {

// polar_ops.cuh as a string (generated by the build from the header itself).
const char kOpsSource[] =
#include "polar_ops_embed.inc"
    ;

// NVRTC, resolved at run time so the library loads on machines without it.
struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

const Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *name : names)
            if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
        n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
        n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
        n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.log_size && n.log && n.destroy;
    });
    return n;
}

// The driver calls used on compiled decoders, looked up through the runtime
// (no link dependency on libcuda).
struct Driver {
    decltype(&cuKernelGetFunction) kernel_get_function = nullptr;
    decltype(&cuFuncGetAttribute) func_get_attribute = nullptr;
    decltype(&cuFuncSetAttribute) func_set_attribute = nullptr;
    decltype(&cuOccupancyMaxActiveBlocksPerMultiprocessor) occupancy = nullptr;
    decltype(&cuLaunchKernel) launch = nullptr;
    bool ok = false;
};

const Driver &driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto get = [](const char *name, void **fp) {
            cudaDriverEntryPointQueryResult q{};
            return cudaGetDriverEntryPointByVersion(name, fp, 12000, cudaEnableDefault, &q) ==
                       cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *fp;
        };
        d.ok = get("cuKernelGetFunction", reinterpret_cast<void **>(&d.kernel_get_function)) &&
               get("cuFuncGetAttribute", reinterpret_cast<void **>(&d.func_get_attribute)) &&
               get("cuFuncSetAttribute", reinterpret_cast<void **>(&d.func_set_attribute)) &&
               get("cuOccupancyMaxActiveBlocksPerMultiprocessor",
                   reinterpret_cast<void **>(&d.occupancy)) &&
               get("cuLaunchKernel", reinterpret_cast<void **>(&d.launch));
        if (!d.ok) cudaGetLastError();
    });
    return d;
}

// CUfunction of a compiled decoder in the current device's context, with its
// dynamic shared-memory limit raised to the device maximum (cached per device).
CUfunction device_function(CompiledKernel *ck) {
    const Driver &drv = driver();
    if (!drv.ok) return nullptr;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    auto it = ck->func.find(device);
    if (it != ck->func.end()) return static_cast<CUfunction>(it->second);
    cudaFree(nullptr);  // make the primary context current
    CUfunction f = nullptr;
    if (drv.kernel_get_function(&f, reinterpret_cast<CUkernel>(ck->kernel)) != CUDA_SUCCESS) return nullptr;
    // The dynamic limit plus the kernel's static shared memory may not exceed
    // the opt-in maximum per block.
    int optin = 0, static_smem = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (drv.func_get_attribute(&static_smem, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, f) != CUDA_SUCCESS)
        return nullptr;
    if (drv.func_set_attribute(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                               optin - static_smem) != CUDA_SUCCESS)
        return nullptr;
    ck->func[device] = f;
    return f;
}

const char *kind_name(uint32_t kind) {
    static const char *names[] = {"polar::OP_F", "polar::OP_G", "polar::OP_G0R"};
    return names[kind];
}

}  // namespace

namespace {

// struct <name> { operator()(frame) }: the code's operation list with every
// node size and offset written as a constant. S = shared-memory stage cap,
// W = widest node run on warp 0 alone, R = largest register-resident subtree.
// ops[i..i+4] are F, Repetition, G, SPC, Combine of one node of 8 or 16 leaves,
// all inside one register subtree (Sec. II-D, "Repetition-SPC codes").
bool is_repspc(const std::vector<HostOp> &ops, size_t i) {
    if (i + 4 >= ops.size()) return false;
    const HostOp &f = ops[i], &r = ops[i + 1], &g = ops[i + 2], &s = ops[i + 3], &c = ops[i + 4];
    const uint32_t l = f.log2n;
    if (f.kind != OP_F || (l != 3 && l != 4)) return false;
    for (size_t k = i; k <= i + 4; ++k) {
        if (!(ops[k].flags & OPW_REG)) return false;
        if (k > i && (ops[k].flags & OPW_REG_ENTER)) return false;
        if (k < i + 4 && (ops[k].flags & OPW_REG_EXIT)) return false;
    }
    return r.kind == OP_REP && r.log2n == l - 1 && r.off == f.off && g.kind == OP_G &&
           g.log2n == l && g.off == f.off && s.kind == OP_SPC && s.log2n == l - 1 &&
           s.off == f.off + (1u << (l - 1)) && c.kind == OP_C && c.log2n == l && c.off == f.off;
}

// The register-subtree operation i (inside a subtree entered at o0 with n0
// leaves) as a RegSub call; returns the number of list entries it covers
// (5 for a fused Repetition-SPC node).
size_t emit_reg_op(std::ostream &o, const std::vector<HostOp> &ops, size_t i, uint32_t o0,
                   const char *indent) {
    const HostOp &op = ops[i];
    const uint32_t n = 1u << op.log2n, p = op.off - o0;
    if (is_repspc(ops, i)) {  // F, rep, G, spc, combine of one 8- or 16-leaf node
        o << indent << "r.template repspc<" << n << "u, " << p << "u>();\n";
        return 5;
    }
    o << indent << "r.template ";
    switch (op.kind) {
    case OP_F:
    case OP_G:
    case OP_G0R: o << "fg<" << kind_name(op.kind) << ", " << n << "u, " << p << "u>();\n"; break;
    case OP_C: o << "combine<" << n << "u, " << p << "u, false>();\n"; break;
    case OP_C0R: o << "combine<" << n << "u, " << p << "u, true>();\n"; break;
    case OP_R0: o << "r0<" << n << "u, " << p << "u>();\n"; break;
    case OP_R1: o << "r1<" << n << "u, " << p << "u>();\n"; break;
    case OP_REP: o << "rep<" << n << "u, " << p << "u>();\n"; break;
    default: o << "spc<" << n << "u, " << p << "u>();\n"; break;
    }
    return 1;
}

// In the per-lane form (kLocalLeaves), a split node of 4 to 16 leaves inside a
// register subtree is decoded by every lane on its own (RegSub::lenter, lfg,
// lr1, lrep, lspc; Combine and Rate-0 are the same word operations). If
// operation i starts such a node, emits the node's operations in that form and
// returns how many list entries it covered; otherwise 0.
size_t emit_local_node(std::ostream &o, const std::vector<HostOp> &ops, size_t i, uint32_t o0,
                       const char *indent) {
    const HostOp &a = ops[i];
    const uint32_t n = 1u << a.log2n;
    if ((a.kind != OP_F && a.kind != OP_G0R) || n > 16 || n < 4 || (a.flags & OPW_REG_ENTER))
        return 0;
    size_t j = i + 1;  // the node's operations: offsets inside [off, off + n), sizes <= n
    while (j < ops.size() && (ops[j].flags & OPW_REG) && !(ops[j].flags & OPW_REG_ENTER) &&
           ops[j].off >= a.off && ops[j].off < a.off + n && ops[j].log2n <= a.log2n)
        ++j;
    for (size_t k = i; k < j; ++k)
        if (ops[k].flags & OPW_REG_EXIT) return 0;  // the node is the subtree itself
    o << indent << "r.template lenter<" << n << "u>();\n";
    for (size_t k = i; k < j; ++k) {
        const HostOp &op = ops[k];
        const uint32_t m = 1u << op.log2n, p = op.off - o0;
        o << indent << "r.template ";
        switch (op.kind) {
        case OP_F:
        case OP_G:
        case OP_G0R: o << "lfg<" << kind_name(op.kind) << ", " << m << "u, " << p << "u>();\n"; break;
        case OP_C: o << "combine<" << m << "u, " << p << "u, false>();\n"; break;
        case OP_C0R: o << "combine<" << m << "u, " << p << "u, true>();\n"; break;
        case OP_R0: o << "r0<" << m << "u, " << p << "u>();\n"; break;
        case OP_R1: o << "lr1<" << m << "u, " << p << "u>();\n"; break;
        case OP_REP: o << "lrep<" << m << "u, " << p << "u>();\n"; break;
        default: o << "lspc<" << m << "u, " << p << "u>();\n"; break;
        }
    }
    return j - i;
}

// One register-subtree operation (or a per-lane node, or a fused
// Repetition-SPC node) at list index i; returns the entries covered.
size_t emit_reg_ops(std::ostream &o, const std::vector<HostOp> &ops, size_t i, uint32_t o0,
                    const char *indent, bool local) {
    if (local) {
        const size_t used = emit_local_node(o, ops, i, o0, indent);
        if (used) return used;
    }
    return emit_reg_op(o, ops, i, o0, indent);
}

// Compact form: one out-of-line function per distinct register subtree (the
// operations with offsets relative to the subtree, so equal frozen patterns
// share code), emitted before the body; returns, per list index of a subtree's
// first operation, the function's id.
// shared: one id map for several bodies (the mixed-batch kernel), so that equal
// subtrees of different codes share one function; nullptr for a map of its own.
std::map<size_t, size_t> emit_subtree_functions(std::ostringstream &o, const std::vector<HostOp> &ops,
                                                const char *T, uint32_t R,
                                                const std::string &prefix, bool local,
                                                std::map<std::string, size_t> *shared = nullptr) {
    std::map<std::string, size_t> own;
    std::map<std::string, size_t> &ids = shared ? *shared : own;
    std::map<size_t, size_t> at;
    for (size_t i = 0; i < ops.size(); ++i) {
        if (!(ops[i].flags & OPW_REG_ENTER)) continue;
        const uint32_t o0 = ops[i].off, n0 = 1u << ops[i].log2n;
        std::ostringstream b;
        for (size_t j = i;;) {
            const size_t used = emit_reg_ops(b, ops, j, o0, "  ", local);
            j += used;
            if (ops[j - 1].flags & OPW_REG_EXIT) break;
        }
        const std::string key = std::to_string(n0) + "|" + std::to_string(R) + "|" + b.str();
        auto it = ids.find(key);
        if (it == ids.end()) {
            const size_t id = ids.size();
            it = ids.emplace(key, id).first;
            o << "__device__ __noinline__ void " << prefix << "sub" << id << "(const " << T
              << " *in, uint32_t *beta, uint32_t o0) {\n"
              << "  RegSub<" << T << ", " << R << "u> r;\n  r.lane = threadIdx.x & 31u;\n"
              << "  r.template enter<" << n0 << "u>(in);\n" << b.str()
              << "  r.template exit<" << n0 << "u>(beta, o0);\n}\n";
        }
        at[i] = it->second;
    }
    return at;
}

// The stage (node size) an operation outside the register subtrees reads its
// LLRs from, or 0 (Combine, Rate-0 and register operations read none).
uint32_t mem_input_stage(const HostOp &op) {
    if (op.flags & OPW_REG) return 0;
    switch (op.kind) {
    case OP_F: case OP_G: case OP_G0R: case OP_R1: case OP_REP: case OP_SPC: return 1u << op.log2n;
    default: return 0;
    }
}

// The stage an operation writes LLRs to, or 0: F/G/G_0R write stage N_v/2, and
// a Repetition node in memory folds its sum in stage N_v/2.
uint32_t mem_output_stage(const HostOp &op) {
    if (op.flags & OPW_REG) return 0;
    switch (op.kind) {
    case OP_F: case OP_G: case OP_G0R: case OP_REP: return 1u << (op.log2n - 1);
    default: return 0;
    }
}

// L2 prefetches: for an operation that reads a stage held in device memory
// (above S, or the channel when it is read in place), the point where its input
// is fetched ahead of use is the start of the last register subtree before it,
// provided no operation in between rewrites that stage (the subtree's work then
// covers the fetch latency). Returns, per list index, the stages to prefetch
// there.
std::vector<std::vector<uint32_t>> plan_prefetch(const std::vector<HostOp> &ops, uint32_t N,
                                                 uint32_t S, bool chan_global) {
    std::vector<std::vector<uint32_t>> at(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        const uint32_t n = mem_input_stage(ops[i]);
        if (!n || !((n == N && chan_global) || (n < N && n > S))) continue;
        for (size_t j = i; j-- > 0;) {
            if (mem_output_stage(ops[j]) == n) break;  // produced since: still in L2
            if (ops[j].flags & OPW_REG_ENTER) {
                at[j].push_back(n);
                break;
            }
        }
    }
    return at;
}

// warp_frames: the body for several frames per CTA, one per warp (run by
// run_warp_frames): every operation is warp-level on the warp's own frame, and
// a CTA barrier after each register subtree keeps the warps in step.
// chan_global: the channel LLRs are read in place from device memory.
// shared_subs: emit register-subtree functions into one map shared with other
// bodies, named with the prefix "Shared_" (see emit_subtree_functions).
void emit_body(std::ostringstream &o, const polar_code &code, bool is_i8, uint32_t S, uint32_t W,
               uint32_t R, const std::string &name, uint32_t outline = 0,
               bool warp_frames = false, bool chan_global = true,
               std::map<std::string, size_t> *shared_subs = nullptr) {
    const bool outline_sub = outline & kOutlineSubtrees, outline_mem = outline & kOutlineMemory;
    const bool local = outline & kLocalLeaves;
    const uint32_t N = code.N;
    const std::vector<HostOp> ops = code.build_ops(R);
    const std::vector<std::vector<uint32_t>> prefetch = plan_prefetch(ops, N, S, chan_global);
    const uint32_t es = is_i8 ? 1u : 4u;
    // last[i]: operation i is the last to read its input stage before an
    // operation rewrites it (a register subtree's entry reads its root stage)
    auto reads = [&](size_t j) -> uint32_t {
        return (ops[j].flags & OPW_REG_ENTER) ? (1u << ops[j].log2n) : mem_input_stage(ops[j]);
    };
    std::vector<bool> last(ops.size(), false);
    for (size_t i = 0; i < ops.size(); ++i) {
        const uint32_t n = reads(i);
        if (!n || n == N) continue;  // the channel is never rewritten
        bool more = false;
        for (size_t j = i + 1; j < ops.size(); ++j) {
            if (reads(j) == n) { more = true; break; }
            if (mem_output_stage(ops[j]) == n) break;
        }
        last[i] = !more;
    }
    auto scratch = [&](uint32_t n) { return n < N && n > S; };
    // how operation i reads its input (RD_*), and whether its input stage is
    // discarded from L2 after it
    auto rd_of = [&](size_t i) -> uint32_t {
        const uint32_t n = reads(i);
        if (n == N && chan_global) return RD_STREAM;
        return (scratch(n) && last[i]) ? RD_LAST : RD_NORMAL;
    };
    auto discard = [&](size_t i, const char *grp, const char *indent) {
        if (rd_of(i) != RD_LAST) return;
        const uint32_t n = reads(i);
        o << indent << "discard_l2<" << grp << ">(gen_in<T, N, S, " << n << "u>(fr), " << n * es
          << "u);\n";
    };
    auto rd_name = [](uint32_t rd) {
        return rd == RD_LAST ? "polar::RD_LAST" : (rd == RD_STREAM ? "polar::RD_STREAM" : "polar::RD_NORMAL");
    };
    const char *T = is_i8 ? "int8_t" : "float";
    std::map<size_t, size_t> sub_at;
    const std::string sub_prefix = shared_subs ? std::string("Shared_") : name + "_";
    if (outline_sub) sub_at = emit_subtree_functions(o, ops, T, R, sub_prefix, local, shared_subs);
    o << "struct " << name << " {\n"
      << "  __device__ __forceinline__ void operator()(const Frame<" << T << "> &fr, float *) const {\n"
      << "    using T = " << T << ";\n"
      << "    constexpr uint32_t N = " << N << "u, S = " << S << "u;\n"
      << "    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;\n"
      << "    (void)lane; (void)warp;\n";

    auto in = [&](uint32_t n) {
        std::ostringstream s;
        s << "gen_in<T, N, S, " << n << "u>(fr)";
        return s.str();
    };
    auto out = [&](uint32_t n) {
        std::ostringstream s;
        s << "gen_out<T, S, " << n << "u>(fr)";
        return s.str();
    };
    // Memory-resident operation on the whole CTA or on warp 0 (inlined with
    // constant arguments: out-of-line copies measured slower).
    auto mem_op = [&](size_t idx, const char *grp) {
        const HostOp &op = ops[idx];
        const uint32_t n = 1u << op.log2n, off = op.off;
        const char *rd = rd_name(rd_of(idx));
        if (outline_mem) {  // out-of-line calls with run-time sizes
            switch (op.kind) {
            case OP_F:
            case OP_G:
            case OP_G0R:
                o << "      mem_fg<T, " << grp << ", " << kind_name(op.kind) << ", " << rd << ">("
                  << in(n) << ", " << out(n / 2) << ", " << n / 2 << "u, fr.beta, " << off << "u);\n";
                break;
            case OP_C:
            case OP_C0R:
                o << "      mem_combine<" << grp << ">(fr.beta, " << n << "u, " << off << "u, "
                  << (op.kind == OP_C0R ? "true" : "false") << ");\n";
                break;
            case OP_R0: o << "      mem_r0<" << grp << ">(fr.beta, " << n << "u, " << off << "u);\n"; break;
            case OP_R1:
                o << "      mem_r1<T, " << grp << ">(" << in(n) << ", fr.beta, " << n << "u, " << off
                  << "u);\n";
                break;
            case OP_REP:
                o << "      mem_rep<T, " << grp << ">(" << in(n) << ", " << out(n / 2) << ", fr.beta, "
                  << n << "u, " << off << "u);\n";
                break;
            default:
                o << "      mem_spc<T, " << grp << ">(" << in(n) << ", fr.beta, " << n << "u, " << off
                  << "u, fr.rkey, fr.rpar);\n";
                break;
            }
            return;
        }
        switch (op.kind) {
        case OP_F:
        case OP_G:
        case OP_G0R:
            o << "      op_fg<T, " << grp << ", " << kind_name(op.kind) << ", " << rd << ">("
              << in(n) << ", " << out(n / 2) << ", " << n / 2 << "u, fr.beta, " << off << "u);\n";
            break;
        case OP_C:
        case OP_C0R:
            o << "      op_combine<" << grp << ">(fr.beta, " << n << "u, " << off << "u, "
              << (op.kind == OP_C0R ? "true" : "false") << ");\n";
            break;
        case OP_R0:
            o << "      op_r0<" << grp << ">(fr.beta, " << n << "u, " << off << "u);\n";
            break;
        case OP_R1:
            o << "      op_r1<T, " << grp << ">(" << in(n) << ", fr.beta, " << n << "u, " << off
              << "u);\n";
            break;
        case OP_REP:
            o << "      op_rep<T, " << grp << ">(" << in(n) << ", " << out(n / 2) << ", fr.beta, "
              << n << "u, " << off << "u);\n";
            break;
        default:
            o << "      op_spc<T, " << grp << ">(" << in(n) << ", fr.beta, " << n << "u, " << off
              << "u, fr.rkey, fr.rpar);\n";
            break;
        }
    };

    // Memory-resident F/G/G_0R operation i followed by up to max_chain - 1
    // operations that each read the stage the previous one wrote (the first
    // operation of the node it produced LLRs for: F or G_0R): emitted as one
    // fused op_chain when the last stage holds at least one vector per column.
    // Returns the number of operations covered (1 = not fused). int8 chains stop
    // at two operations: three hold eight 16-byte input vectors, which under the
    // 72-register budget of the int8 decoder means more local memory, and they
    // measured slower (with byte-wise and with f16 arithmetic alike); float32
    // chains go to three.
    const uint32_t vec = is_i8 ? 16u : 4u;
    const uint32_t max_chain = is_i8 ? 2u : 3u;
    auto chain_len = [&](size_t i) -> uint32_t {
        const HostOp &a = ops[i];
        if ((a.flags & OPW_REG) || a.kind > OP_G0R) return 1;
        uint32_t len = 1;
        for (size_t j = i; len < max_chain && j + 1 < ops.size(); ++j, ++len) {
            const HostOp &p = ops[j], &q = ops[j + 1];
            const uint32_t pn = 1u << p.log2n;
            const uint32_t child_off = p.kind == OP_F ? p.off : p.off + pn / 2;
            if ((q.flags & OPW_REG) || (q.kind != OP_F && q.kind != OP_G0R) ||
                q.log2n + 1 != p.log2n || q.off != child_off)
                break;
        }
        while (len > 1 && ((1u << a.log2n) >> len) < vec) --len;
        return len;
    };
    auto chain_op = [&](size_t i, uint32_t len, const char *grp) {
        const HostOp &a = ops[i];
        const uint32_t n = 1u << a.log2n;
        // an intermediate stage whose only reader is the next operation of the
        // chain is not stored
        const uint32_t store = (last[i + 1] ? 0u : 1u) | (len == 3 && last[i + 2] ? 0u : 2u);
        o << "      " << (outline_mem ? "mem_chain" : "op_chain") << "<T, " << grp << ", " << len
          << "u, " << kind_name(a.kind) << ", " << kind_name(ops[i + 1].kind) << ", "
          << (len == 3 ? kind_name(ops[i + 2].kind) : "polar::OP_F") << ", " << store << "u, "
          << rd_name(rd_of(i)) << ">(" << in(n) << ", " << out(n / 2) << ", " << out(n / 4) << ", "
          << (len == 3 ? out(n / 8) : "nullptr") << ", " << n << "u, fr.beta, " << a.off << "u);\n";
    };

    bool in_run = false;
    uint32_t o0 = 0, n0 = 0;
    for (size_t i = 0; i < ops.size(); ++i) {
        const HostOp &op = ops[i];
        const uint32_t n = 1u << op.log2n;
        const bool narrow = warp_frames || n <= W || (op.flags & OPW_REG);
        const uint32_t clen = chain_len(i);
        if (!narrow) {
            if (in_run) {
                o << "    }\n    __syncthreads();\n";
                in_run = false;
            }
            o << "    {\n";
            if (clen > 1) chain_op(i, clen, "CtaGrp");
            else mem_op(i, "CtaGrp");
            o << "    }\n    __syncthreads();\n";
            discard(i, "CtaGrp", "    ");
            i += clen - 1;
            continue;
        }
        if (!in_run) {
            o << (warp_frames ? "    {\n" : "    if (warp == 0) {\n");
            in_run = true;
        }
        if (!(op.flags & OPW_REG) && clen > 1) {
            chain_op(i, clen, "WarpGrp");
            o << "      __syncwarp();\n";
            discard(i, "WarpGrp", "      ");
            i += clen - 1;
            continue;
        }
        if (!(op.flags & OPW_REG)) {
            mem_op(i, "WarpGrp");
            o << "      __syncwarp();\n";
            discard(i, "WarpGrp", "      ");
            continue;
        }
        const char *align = warp_frames ? "      __syncthreads();\n" : "";
        for (uint32_t pn : prefetch[i])
            o << "      prefetch_l2(" << in(pn) << ", " << pn * es << "u);\n";
        if (outline_sub && (op.flags & OPW_REG_ENTER)) {  // the whole subtree is one call
            o << "      " << sub_prefix << "sub" << sub_at.at(i) << "(" << in(n) << ", fr.beta, " << op.off
              << "u);\n      __syncwarp();\n" << align;
            while (!(ops[i].flags & OPW_REG_EXIT)) ++i;
            continue;
        }
        if (op.flags & OPW_REG_ENTER) {
            o0 = op.off;
            n0 = n;
            o << "      {\n        RegSub<T, " << R << "u> r;\n        r.lane = lane;\n"
              << "        r.template enter<" << n0 << "u>(" << in(n0) << ");\n";
        }
        i += emit_reg_ops(o, ops, i, o0, "        ", local) - 1;
        if (ops[i].flags & OPW_REG_EXIT) {
            o << "        r.template exit<" << n0 << "u>(fr.beta, " << o0 << "u);\n      }\n"
              << "      __syncwarp();\n" << align;
        }
    }
    if (in_run) o << "    }\n" << (warp_frames ? "    __syncwarp();\n" : "    __syncthreads();\n");
    o << "  }\n};\n";
}

}  // namespace

std::string generate_source(const polar_code &code, bool is_i8, const LaunchShape &shape,
                            uint32_t reg_subtree, uint32_t outline) {
    std::ostringstream o;
    o << "// Fast-SSC decoder specialised to one (" << code.N << ", " << code.K << ") polar code"
      << ((outline & kOutlineSubtrees) ? ", subtrees out of line" : "")
      << ((outline & kOutlineMemory) ? ", memory operations out of line" : "") << "\n"
      << "#include \"polar_ops.cuh\"\n"
      << "namespace polar {\n";
    const bool warp_frames = shape.frames_per_cta > 1;
    emit_body(o, code, is_i8, shape.smem_stage_max, shape.warp_stage_max, reg_subtree, "GenBody",
              outline, warp_frames, warp_frames || !shape.stage_channel);
    o << "}  // namespace polar\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << shape.threads << ", "
      << std::max<uint32_t>(shape.ctas_per_sm, 1) << ") polar_unrolled(const polar::KernelArgs a) {\n";
    if (warp_frames)
        o << "  polar::run_warp_frames<" << (is_i8 ? "int8_t" : "float") << ">(a, polar::GenBody{});\n}\n";
    else
        o << "  polar::run_frames<" << (is_i8 ? "int8_t" : "float") << ", false, "
          << (shape.stage_channel ? "true" : "false") << ">(a, polar::GenBody{});\n}\n";
    return o.str();
}

std::string generate_batch_source(const std::vector<const polar_code *> &codes, bool is_i8,
                                  const std::vector<uint32_t> &S, const std::vector<uint32_t> &W,
                                  const std::vector<uint32_t> &R, uint32_t threads,
                                  uint32_t min_blocks, uint32_t outline, bool warp_frames) {
    std::ostringstream o;
    const char *T = is_i8 ? "int8_t" : "float";
    o << "// Mixed-batch Fast-SSC decoder: one specialised body per code\n"
      << "#include \"polar_ops.cuh\"\n"
      << "namespace polar {\n";
    std::map<std::string, size_t> shared;  // subtree functions common to every body
    for (size_t c = 0; c < codes.size(); ++c)
        emit_body(o, *codes[c], is_i8, S[c], W[c], R[c], "Body" + std::to_string(c), outline,
                  warp_frames, true, &shared);
    o << "struct BatchBody {\n"
      << "  __device__ __forceinline__ void operator()(uint32_t cid, const Frame<" << T
      << "> &fr) const {\n    switch (cid) {\n";
    for (size_t c = 0; c < codes.size(); ++c)
        o << "    case " << c << ": Body" << c << "{}(fr, nullptr); break;\n";
    o << "    default: break;\n    }\n  }\n};\n}  // namespace polar\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << threads << ", "
      << std::max<uint32_t>(min_blocks, 1) << ") polar_batch(const polar::BatchArgs a) {\n"
      << "  polar::" << (warp_frames ? "run_batch_warps<" : "run_batch<") << T
      << ">(a, polar::BatchBody{});\n}\n";
    return o.str();
}

cudaError_t compile_source(const std::string &src, CompiledKernel *out, std::string *log,
                           const char *kernel_name) {
    const Nvrtc &nv = nvrtc();
    if (!nv.ok) {
        *log = "NVRTC (libnvrtc.so) could not be loaded";
        return cudaErrorNotSupported;
    }
    int device = 0, major = 0, minor = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    if (e != cudaSuccess) return e;
    char arch[64];
    std::snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%d%s", major, minor, major >= 9 ? "a" : "");

    nvrtcProgram prog = nullptr;
    const char *hdr_src[] = {kOpsSource};
    const char *hdr_name[] = {"polar_ops.cuh"};
    if (nv.create(&prog, src.c_str(), "polar_unrolled.cu", 1, hdr_src, hdr_name) != NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return cudaErrorInvalidValue;
    }
    const char *opts[] = {arch, "-std=c++17", "-default-device", "--ptxas-options=-v"};
    const nvrtcResult r = nv.compile(prog, 4, opts);
    size_t ls = 0;
    nv.log_size(prog, &ls);
    std::string lg(ls, '\0');
    if (ls) nv.log(prog, &lg[0]);
    lg.resize(std::strlen(lg.c_str()));  // drop the terminating NUL
    *log = lg;
    if (r != NVRTC_SUCCESS) {
        nv.destroy(&prog);
        return cudaErrorInvalidSource;
    }
    size_t cs = 0;
    nv.cubin_size(prog, &cs);
    std::vector<char> cubin(cs);
    nv.cubin(prog, cubin.data());
    nv.destroy(&prog);
    e = cudaLibraryLoadData(&out->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return e;
    e = cudaLibraryGetKernel(&out->kernel, out->lib, kernel_name);
    if (e != cudaSuccess) {
        cudaLibraryUnload(out->lib);
        out->lib = nullptr;
        return e;
    }
    CUfunction f = device_function(out);
    if (!f) {
        cudaLibraryUnload(out->lib);
        out->lib = nullptr;
        *log += "\ncould not obtain the compiled kernel's function handle";
        return cudaErrorInvalidDeviceFunction;
    }
    int regs = 0, local = 0, maxt = 0;
    driver().func_get_attribute(&regs, CU_FUNC_ATTRIBUTE_NUM_REGS, f);
    driver().func_get_attribute(&local, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, f);
    driver().func_get_attribute(&maxt, CU_FUNC_ATTRIBUTE_MAX_THREADS_PER_BLOCK, f);
    char line[256];
    std::snprintf(line, sizeof line,
                  "\nkernel: %d registers, %d bytes local, %d max threads, cubin %zu bytes\n",
                  regs, local, maxt, cs);
    *log += line;
    return cudaSuccess;
}

int compiled_max_ctas(CompiledKernel *ck, uint32_t threads, size_t smem_bytes) {
    CUfunction f = device_function(ck);
    if (!f) return 0;
    int n = 0;
    if (driver().occupancy(&n, f, static_cast<int>(threads), smem_bytes) != CUDA_SUCCESS) return 0;
    return n;
}

cudaError_t launch_compiled(CompiledKernel *ck, const LaunchShape &shape, const void *args,
                            cudaStream_t stream) {
    CUfunction f = device_function(ck);
    if (!f) return cudaErrorInvalidDeviceFunction;
    void *params[] = {const_cast<void *>(args)};
    const CUresult r = driver().launch(f, shape.grid, 1, 1, shape.threads, 1, 1,
                                       static_cast<unsigned>(shape.smem_bytes),
                                       reinterpret_cast<CUstream>(stream), params, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

}  // namespace polar
