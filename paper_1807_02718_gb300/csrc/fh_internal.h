// Internal declarations of libfh: device-side parameter blocks and kernel
// launchers.  Host library code (fh_api.cu) owns all state; the kernels only
// see plain pointers and sizes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "fh.h"

namespace fh {

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device.  The attribute lives in each device's context, so
// a process with contexts on several GPUs needs it on every one; `done` holds
// one bit per device (devices beyond 63 set it on every call).  Concurrent
// first calls from several host threads only repeat the (idempotent) call.
inline cudaError_t ensure_smem_attr(const void *fn, int bytes,
                                    std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;

// Obstacle parameters passed by value to the geometry kernel.
struct CurveParams {
    int kind;
    int n_harm;
    double r0;
    double cx, cy;
    double amp[FH_MAX_HARMONICS];
    double phase[FH_MAX_HARMONICS];
};

// Per-solve tables (one entry per frequency with omega > 0).
struct SolveTables {
    const int *N;            // boundary size N_s (= 2 n_s)
    const long long *mat_off;// element offset of matrix s (N_s^2 complex)
    const int *vec_off;      // element offset of node data / density of s
    const int *tab;          // index of the Kress / log-sin table for N_s
    const int *tab_off;      // element offset of table t
    const double *kappa;     // kappa_s = omega_s / c
    const double *eta;       // CFIE coupling eta_s
};

// ---- geometry and quadrature tables (k_geometry.cu) ----
// Solve s uses curve curves[prob[s]] (device arrays).
// zf, dzf: double-float copies of z, z' (x hi, x lo, y hi, y lo); sf: |z'|.
void launch_geometry(const CurveParams *curves, const int *prob, int S, int maxN, const int *N,
                     const int *vec_off, double2 *z, double2 *dz, double2 *ddz, float4 *zf,
                     float4 *dzf, float2 *sf, cudaStream_t st);
// wpf: ((pi/n) ln(4 sin^2(pi d/N)) - R_d) / pi as double-float pairs.
void launch_kress_tables(int n_tab, int maxN, const int *tab_N, const int *tab_off,
                         double *kress, double *logsin, float2 *wpf, cudaStream_t st);

// Frequency subgroups: up to kGroup consecutive solves with equal N (hence
// identical nodes).  Their kernels share the geometry of each node pair and
// advance e^{i kappa_j r} from one frequency to the next by a complex product
// instead of a sincos per frequency.
constexpr int kGroup = 8;
struct Subgroups {
    const int2 *sg;            // (first solve s0, count) per subgroup
    const long long *tile_off; // assembly tiles, prefix over subgroups
    const double *dkappa;      // mean kappa step inside each subgroup
};

// ---- CFIE assembly (k_assemble.cu) ----
// Matrices are column-major: A_s(i, l) = A[mat_off[s] + l * N_s + i].
// Grouped assembly: every matrix of subgroup g at A + mat_off[s] + out_shift.
// Exactly one of A (FP64 complex) and Af (mixed paths: double-float pairs re
// hi, re lo, im hi, im lo, same 16 bytes per entry) is non-null.
// Launches the tiles tile_base .. tile_base + n_tiles - 1 of the subgroup
// table g (n_groups subgroups, tile offsets over the whole table; a matrix of
// order n has ceil(n/32)^2 tiles for A, the ceil(n/32) (ceil(n/32) + 1) / 2
// tiles of its upper triangle for Af).  Mixed
// paths (Af): also the near-diagonal band of the band_count solves in the
// device list band_list (largest N maxN), a second launch, issued first on
// band_st (which may be st; the two kernels write disjoint entries, so that on
// another stream the FP64-bound band overlaps the FP32-bound tiles).  A32
// (mixed paths, may be null): the hi parts of every entry also into the
// row-major FP32 copy of the tensor-core LU (what launch_convert_rowmajor
// would make from Af).
void launch_assemble_groups(const SolveTables &t, const Subgroups &g, int n_groups,
                            long long tile_base, long long n_tiles, const int *band_list,
                            int band_count, int maxN,
                            const double2 *z, const double2 *dz,
                            const double2 *ddz, const double *kress, const double *logsin,
                            const float4 *zf, const float4 *dzf, const float2 *sf, const float2 *wpf,
                            double2 *A, float4 *Af, float2 *A32, long long out_shift, cudaStream_t st,
                            cudaStream_t band_st);
// Solve s uses the incidence direction pdir[prob[s]].
void launch_rhs(const SolveTables &t, int S, int maxN, const double2 *z, const double2 *dz,
                const int *prob, const double2 *pdir, double2 *g, cudaStream_t st);

// ---- batched dense LU with partial pivoting and solve (k_lu.cu) ----
// Solves A_s x = b_s in place (b_s overwritten by x_s); A_s overwritten by
// its LU factors.  order[] lists solves largest first.  info[s] = 0 on
// success, else 1 + column of the first zero / non-finite pivot.
void launch_lu_solve_fp64(const int *order, int S, const int *N, const long long *mat_off,
                          const int *vec_off, double2 *A, double2 *b, int *info, cudaStream_t st);

// Mixed precision: FP32 copy (the hi parts) of the double-float matrices,
// FP32 LU, double-float residual refinement.
void launch_convert_fp32(const float4 *Af, float2 *A32, long long n, cudaStream_t st);
// piv (per system, length N) holds the inverse row permutation on return.
void launch_lu_factor_fp32(const int *order, int S, const int *N, const long long *mat_off,
                           float2 *A32, int *piv, const int *vec_off, int *info, int maxN,
                           cudaStream_t st);
// Tensor-core LU of the row-major FP32 copy (launch_convert_rowmajor); kind 2:
// 3xTF32 operands, kind 1: 3xBF16.  order_h / N_h: host copies of order (by
// decreasing N) and N, used to launch each cluster size separately.  A system
// of order N is factored by the smallest power of two of CTAs, at most 8, that
// is >= N / rows_per_cta (rows_per_cta 128, 256 or 512; 512 gives 1, 2, 4, 8
// CTAs for N <= 512, 1024, 2048, 4096).  err is set and info[s] = -2 if a
// tensor-core completion wait gave up.
constexpr int kTcMaxN = 4096;
int lu_tc_cluster(int n, int rows_per_cta);
int lu_tc_launches(const int *order_h, const int *N_h, int S, int rows_per_cta);
// Row-major FP32 copies of the count solves in the device list list.
void launch_convert_rowmajor(const int *list, int count, const int *N, const long long *mat_off,
                             const float4 *Af, float2 *A32, cudaStream_t st);
// Work space of the tensor-core LU (indexed by solve, like N and mat_off):
// maps: S tensor maps of the row-major FP32 matrices (lu_tc_encode_maps,
// copied to the device); opnd: the staged operand tiles of every system,
// system s's L21 tiles at byte a_off[s] and U12 tiles at b_off[s]
// (lu_tc_opnd_bytes fills host copies of the offsets and returns the size).
struct LuTcWork {
    const void *maps;
    uint8_t *opnd;
    const long long *a_off, *b_off;
};
size_t lu_tc_opnd_bytes(int kind, const int *N_h, int S, long long *a_off_h, long long *b_off_h);
size_t lu_tc_map_bytes(int S);
// Host: encodes the tensor maps of systems 0..S-1 (matrix s at A32 +
// mat_off_h[s], order N_h[s]) into maps_h (lu_tc_map_bytes(S) bytes).
cudaError_t lu_tc_encode_maps(const int *N_h, const long long *mat_off_h, int S, float2 *A32, void *maps_h);
cudaError_t launch_lu_factor_tc(int kind, int rows_per_cta, const int *order, const int *order_h,
                                const int *N_h, int S,
                                const int *N, const long long *mat_off, float2 *A32, int *piv,
                                const int *vec_off, int *info, int *err, const LuTcWork &w,
                                cudaStream_t st);
// Iterative refinement against the column-major double-float matrices Af
// (residuals with exact products and double-float sums); chunks
// lists (solve, first row) per kResidRows rows; state holds
// refine_state_bytes(S) bytes; y32 one FP32 complex per unknown.
constexpr int kResidRows = 64;
size_t refine_state_bytes(int S);
// Row-major factors: blocks lists (solve, 32-row block) for the diagonal-block
// inverses, blk_off the first block of each solve, inv 2048 FP32 complex per
// block (scratch).
void launch_lu_refine(bool row_major, const int *order, int S, const int *N,
                      const long long *mat_off, const int *vec_off, const int2 *chunks,
                      int n_chunks, const int2 *blocks, int n_blocks, const int *blk_off,
                      float2 *inv, const float4 *Af, const float2 *LU32, const int *piv,
                      const double2 *g, double2 *x, float2 *y32, void *state, int max_iters,
                      double tol, int *iters, double *resid, int *info, int maxN, cudaStream_t st);

// ---- window spectra (k_window.cu) ----
void launch_window_spectra(const double *a, int n_samples, long long start0, long long step,
                           int Q, double dt, double H, int K, int J, const double *omega,
                           double *wa_scratch, double2 *B, cudaStream_t st);

// ---- target fields (k_field.cu) ----
// V[j * n_x + i] = V(x_i, omega_j); V[0 * n_x + i] = 1 (omega_0 = 0).
// Work items (subgroup, first node) of `chunk` <= kFieldChunk nodes;
// item_first[g] is the first item of subgroup g (global, one entry past the
// last subgroup).  One problem's subgroups g_begin .. g_begin + n_groups - 1
// own the items item_begin .. item_begin + n_items - 1.  part: scratch of
// n_items * kGroup * n_x complex values.  group_max: the largest subgroup
// size (<= kGroup; the double-float kernel is compiled for 4 and kGroup).
constexpr int kFieldChunk = 64;
void launch_target_field(const SolveTables &t, const Subgroups &g, int g_begin, int n_groups,
                         const int2 *items, int item_begin, int n_items, int chunk,
                         int group_max, const int *item_first, const int *solve_j,
                         const double2 *z, const double2 *dz, const double2 *psi, const double *x,
                         int n_x, const float4 *zf, double2 *part, double2 *V, bool double_float,
                         cudaStream_t st);

// Kernel Bessel routine on n arguments: out[6i..6i+5] = J0, Y0, J1, Y1 (joint
// routine) and J0, Y0 (H0-only routine).
void launch_bessel_eval(const double *x, int n, double *out, cudaStream_t st);
// out[4i..4i+3] = J0, Y0, J1, Y1 through the double-float Hankel form (x >= 8).
void launch_bessel_eval_df(const double *x, int n, double *out, cudaStream_t st);

// ---- synthesis (k_synth.cu) ----
// nu[r * J + p] = sum_{m=-h}^{h-1} (-1)^m T_r(m/h) e^{-2 pi i m p / M} (T_r
// the Chebyshev polynomials, the r = 0 row halved; nu may be null), and nu_f
// the same as double-float pairs (re hi, re lo, im hi, im lo); pw is scratch
// of M * kFarTerms doubles.  Far windows (|y| >= 1.25 h) need at most 48 terms.
constexpr int kFarTerms = 64;
void launch_far_table(int J, int M, double *pw, double2 *nu, float4 *nu_f, float4 *phase_tab,
                      cudaStream_t st);
// Gr/Gm: planes [p][t] with u(x,t) = sum_p Vr[p][x] Gr[p][t] + Vi[p][x] Gm[p][t].
// Gs (optional; then Gr/Gm are not written): the same weights as double-float
// pairs (hi, lo), rows p = Gr[p] and J + p = Gm[p], row pitch synth_pitch(n_T),
// for launch_synth_contract_df.  Bf: optional scratch of K * J float4 for the
// double-float copy of B (one extra launch); null splits B on the fly.
inline int synth_pitch(int n) { return (n + 3) & ~3; }
void launch_synth_weights(int J, int M, double W, int K, const double *s, const double2 *B,
                          float4 *Bf, const float4 *nu_f, const float4 *phase_tab,
                          const float4 *sinc_tab, const double *T, int n_T, double *Gr, double *Gm,
                          float2 *Gs, cudaStream_t st);
// Dynamic shared memory launch_synth_weights needs for J frequencies and K
// windows, with (`table`) or without the near-sum table; at most
// kWeightsMaxSmem bytes are available (so K and J are bounded; callers
// reject larger problems before launching).
constexpr size_t kWeightsMaxSmem = 200 * 1024;
size_t synth_weights_smem(int J, int K, bool table);
// Near-window sums by interpolation.  The near sums
//   D_p(y) = sum_{m=-h}^{h-1} e^{-2 pi i m p / M} sinc(y - m)
// are, as functions of y, band-limited to [-pi, pi]; sampled on the
// half-integer grid y_g = g / 2 (oversampling 2) they are recovered by
//   D_p(y) = sum_g D_p(y_g) sinc(2 (y - y_g)) E(y - y_g),
// E(u) = exp(beta (sqrt(1 - (u / U)^2) - 1)) for |u| < U (the "exponential of
// semicircle" window), with U = 10.5 and beta = 32.5: 42 samples per y; the
// window's Fourier transform is flat to 1.4e-15 on [-pi, pi] and its aliases
// from [3 pi, inf) sum below 1.1e-15.  The table holds D_p(y_g) for |g| <= G =
// ceil(2.5 h) + 24 (every near y, |y| < 1.25 h, with its 42 samples) as
// double-float pairs (re hi, re lo, im hi, im lo), row g + G, column p:
// integer rows are the phases themselves, half-integer rows the direct sums
// in double-float.  Built for J <= kSincTabMaxJ (table size (2G + 1) J).
constexpr int kSincTabMaxJ = 1025;
constexpr int kSincPts = 42;
constexpr double kSincU = 10.5;
constexpr double kSincBeta = 32.5;
inline int sinc_tab_half(int J) { return J >= 2 && J <= kSincTabMaxJ ? (5 * (J - 1) + 1) / 2 + 24 : 0; }
inline long long sinc_tab_entries(int J) {
    const int G = sinc_tab_half(J);
    return G ? (2LL * G + 1) * J : 0;
}
void launch_sinc_table(int J, int M, const float4 *phase_tab, float4 *tab, cudaStream_t st);
// FP64 contraction u = [Vr | Vi] [Gr ; Gm] (FP64 FMAs).
void launch_synth_contract(int J, int n_x, int n_T, const double2 *V, const double *Gr,
                           const double *Gm, double *u, cudaStream_t st);
// Tensor-core contraction (mixed-precision paths, 2J <= kContractTcMaxK): the
// operands cut into eight 6-bit slices held exactly in BF16, every slice
// product summed exactly in FP32 per level over K segments of 512, levels and
// segments combined in double-float.
// scratch: contract_tc_scratch_bytes(J, n_x, n_T) bytes; err set if an MMA
// completion wait gave up.  Six launches.
constexpr int kContractTcMaxK = 8192;
bool contract_tc_ok(int J);
size_t contract_tc_scratch_bytes(int J, int n_x, int n_T);
cudaError_t launch_contract_tc(int J, int n_x, int n_T, const double2 *V, const double *Gr,
                               const double *Gm, double *u, void *scratch, int *err, cudaStream_t st);
int contract_tc_kpad(int J);
int contract_tc_rows(int n);
int contract_tc_cols(int n);
// Double-float contraction (mixed-precision paths): V is split into Vs
// (scratch of 2J rows of synth_pitch(n_x) float2), then u = Vs^T Gs with exact
// products and double-float accumulation.  Two launches.
void launch_synth_contract_df(int J, int n_x, int n_T, const double2 *V, float2 *Vs,
                              const float2 *Gs, double *u, cudaStream_t st);

}  // namespace fh
