// Writes the CUDA source that the run-time code generator (polar_codegen.cpp)
// emits for one code and one launch shape, or for a mixed batch of codes, so
// that a host test can compile it for sm_103a with nvcc: the same program that
// polar_code_compile / polar_batch_create hand to NVRTC on a GPU.
//
//   codegen_source code  OUT.cu MASK N K IS_I8 THREADS S W FRAMES_PER_CTA STAGE REG OUTLINE CTAS
//   codegen_source batch OUT.cu IS_I8 THREADS MIN_BLOCKS OUTLINE WARP_FRAMES {MASK N K S W REG}...
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"

static polar_code *load_code(const char *mask_path, uint32_t N, uint32_t K) {
    std::vector<uint8_t> m(N);
    FILE *f = std::fopen(mask_path, "rb");
    if (!f || std::fread(m.data(), 1, N, f) != N) {
        std::printf("cannot read %s\n", mask_path);
        std::exit(2);
    }
    std::fclose(f);
    polar_code_t *c = nullptr;
    const polar_status st = polar_code_create(N, K, m.data(), &c);
    if (st != POLAR_OK) {
        std::printf("polar_code_create: %s\n", polar_status_str(st));
        std::exit(2);
    }
    return reinterpret_cast<polar_code *>(c);
}

static uint32_t u(const char *s) { return static_cast<uint32_t>(std::strtoul(s, nullptr, 10)); }

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    const std::string mode = argv[1];
    std::string src;
    if (mode == "code" && argc == 15) {
        polar_code *c = load_code(argv[3], u(argv[4]), u(argv[5]));
        polar::LaunchShape sh{};
        sh.threads = u(argv[7]);
        sh.smem_stage_max = u(argv[8]);
        sh.warp_stage_max = u(argv[9]);
        sh.frames_per_cta = u(argv[10]);
        sh.stage_channel = u(argv[11]);
        sh.ctas_per_sm = u(argv[14]);
        src = polar::generate_source(*c, u(argv[6]) != 0, sh, u(argv[12]), u(argv[13]));
    } else if (mode == "batch" && argc > 8 && (argc - 8) % 6 == 0) {
        std::vector<const polar_code *> codes;
        std::vector<uint32_t> S, W, R;
        for (int i = 8; i < argc; i += 6) {
            codes.push_back(load_code(argv[i], u(argv[i + 1]), u(argv[i + 2])));
            S.push_back(u(argv[i + 3]));
            W.push_back(u(argv[i + 4]));
            R.push_back(u(argv[i + 5]));
        }
        src = polar::generate_batch_source(codes, u(argv[3]) != 0, S, W, R, u(argv[4]), u(argv[5]),
                                           u(argv[6]), u(argv[7]) != 0);
    } else {
        std::printf("bad arguments\n");
        return 2;
    }
    std::ofstream(argv[2]) << src;
    std::printf("OK %zu\n", src.size());
    return 0;
}
