// Synthesis entry point that allocates no memory.
//
// fh_synthesize_static runs the same synthesis kernels as the context-based
// path (far-field table, weights, contraction), but its scratch (the weight
// planes G and the phase / far-field tables) lives in one file-scope device
// array instead of memory the library allocates.  It is meant for callers
// that may not allocate device memory at the point where they need the field:
// code running inside a real-time or serving loop with a fixed memory budget,
// hosts whose device memory is handed out by their own arena, or callers that
// must not trigger the implicit synchronisation of cudaMalloc / cudaFree.
#include <mutex>

#include "fh_internal.h"

namespace {

// Scratch capacity: J * n_T <= kMaxGridPoints, J <= kMaxJ.
constexpr long long kMaxGridPoints = 1LL << 19;     // G planes: 2 x 8 B x 2^19 = 8 MiB
static_assert(2 * kMaxGridPoints >= 2LL * 2048 * fh::kFarTerms, "power table fits in the G planes");
constexpr int kMaxJ = 2049;                         // M = 2(J-1) <= 4096
constexpr size_t kScratchDoubles = 2 * (size_t)kMaxGridPoints   // Gr, Gm
                                   + 2 * (size_t)fh::kFarTerms * kMaxJ   // far-field table (double-float)
                                   + 2 * (size_t)(2 * (kMaxJ - 1));      // phase table

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_synth_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
fh_status scratch_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FH_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_synth_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FH_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return FH_OK;
}

}  // namespace

extern "C" fh_status fh_synthesize_static(int J, double W, int K, const double *d_s,
                                          const double *d_B, const double *d_V, int n_x,
                                          const double *d_T, int n_T, double *d_u,
                                          void *cuda_stream) {
    if (J < 2 || J > kMaxJ || K < 1 || n_x < 0 || n_T < 0 || !(W > 0.0)) return FH_EINVAL;
    if ((long long)J * n_T > kMaxGridPoints) return FH_EINVAL;
    // the weights kernel keeps per-window arrays and the phase rows in shared memory
    if (fh::synth_weights_smem(J, K, false) > fh::kWeightsMaxSmem) return FH_EINVAL;
    if (n_x == 0 || n_T == 0) return FH_OK;
    if (!d_s || !d_B || !d_V || !d_T || !d_u) return FH_EINVAL;
    // An error left pending by earlier, unrelated work belongs to its owner:
    // report it without launching and without clearing it.
    if (cudaPeekAtLastError() != cudaSuccess) return FH_ECUDA;
    double *scratch = nullptr;
    const fh_status st = scratch_address(&scratch);
    if (st != FH_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const int M = 2 * (J - 1);
    double *Gr = scratch;
    double *Gm = Gr + (size_t)J * n_T;
    double *pw = scratch;   // power table of the far-field table; G is written after it is used
    float4 *nu_f = reinterpret_cast<float4 *>(scratch + 2 * (size_t)kMaxGridPoints);
    float4 *ph = nu_f + (size_t)fh::kFarTerms * kMaxJ;   // phase table, double-float
    fh::launch_far_table(J, M, pw, nullptr, nu_f, ph, stream);
    fh::launch_synth_weights(J, M, W, K, d_s, reinterpret_cast<const double2 *>(d_B), nullptr, nu_f, ph,
                             nullptr, d_T, n_T, Gr, Gm, nullptr, stream);   // direct near sums
    fh::launch_synth_contract(J, n_x, n_T, reinterpret_cast<const double2 *>(d_V), Gr, Gm, d_u, stream);
    return cudaGetLastError() == cudaSuccess ? FH_OK : FH_ECUDA;
}
