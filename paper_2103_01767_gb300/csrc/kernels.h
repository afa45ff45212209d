// kernels.h -- internal interface between the C-ABI host code and the FFT kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace ptylm {

// Arguments shared by the per-position kernels.  Pointers not used by a kernel are NULL.
struct PtyArgs {
    const float2* O;       // object (forward, jtvp, jvp linearisation point) or vector (matvec)
    const float2* V;       // second gathered array: the direction vO of jvp
    const float2* P;       // probe [S][S]
    const int2* pos;       // positions [K] as (row, col)
    const float* y;        // measurements [K][M] in team-register order: sqrt(y) (Gaussian) or y (Poisson)
    const float* w;        // jtvp weights [K][S][S]
    float2* a_cache;       // [K][M] per-pixel factor a, team-register order
    float2* out;           // scatter-add target [ny][nx] (gradient, matvec, jtvp)
    float* out_real;       // jvp output [K][S][S]
    float2* scratch;       // jvp: one M-sized slot per team
    double* partials;      // per-CTA FP64 partial sums [gridDim.x][<=4] (grid_reduce scratch)
    unsigned* counter;     // grid_reduce counter (zero between launches)
    double* scal;          // FP64 scalar slots (reduce.cuh Slot)
    const float2* tw;      // twiddles W_S^j = exp(-2 pi i j / S), j < S
    int K;
    int nx;
    float b;               // background
    int loss;              // 0 Gaussian, 1 Poisson
    const float2* VP;      // joint: probe part of the direction (matvec, jvp)
    const float2* Olin;    // joint: object at the linearisation point (matvec)
    float2* outP_part;     // joint: per-team probe accumulators [grid * TEAMS][M]
    float* trp;            // optional: per-thread sums of d2l [K][T] (forward + cache)
    const double* skip;    // matvec: return at once when *skip != 0 (a CG solve that has converged)
};

enum KernelId {
    KID_FWD_LOSS = 0, KID_FWD_CACHE = 1, KID_MATVEC = 2, KID_JTVP = 3, KID_JVP = 4, KID_FWD_INTENSITY = 5,
    KID_FWD_CACHE_J = 6, KID_MATVEC_J = 7, KID_JTVP_J = 8, KID_JVP_J = 9,
    KID_FWD_MAG = 10,                       // zeta (natural order) and optionally u = psihat / zeta
    KID_JVP_U = 11, KID_JVP_U_J = 12,       // J v from the stored phasor u (one FFT)
    KID_JTVP_U = 13, KID_JTVP_U_J = 14,     // J^T w from the stored phasor u (one FFT)
    KID_COUNT = 15
};

// Closed-form GGN diagonal (App. B, Eqs. ggn_diag_mat and ggn_joint_diag) from the per-thread
// d2l sums of the last linearisation: D_O += |P|^2 tr_k / (2M) over each patch (one CTA per
// position, D_O zeroed first) and, when D_P != NULL, D_P[m] = sum_k |O[r_k + m]|^2 tr_k / (2M).
cudaError_t launch_ggn_diag(int LS, int LE, const float* trp, const int2* pos, int K, const float2* O,
                            const float2* P, int nx, float* D_O, float* D_P, float* tr, cudaStream_t stream);

// FFT tile of a single-problem context: patch side 2^LS with 2^LE values per thread (LE = 5,
// or 4 for sides 32 and 64: teams of S^2/16 threads).  Threads per CTA and teams (positions
// in flight) per CTA for that tile.
int cta_threads(int LS, int LE);
int cta_teams(int LS, int LE);
size_t cta_smem_bytes(int LS, int LE);

// Opt in to the kernel's dynamic shared memory and report how many CTAs fit on one SM.
cudaError_t kernel_prepare(int LS, int LE, int kid, int* ctas_per_sm);

// Copy measurements from natural [K][S][S] order into the kernels' team-register order
// (square roots when take_sqrt: the Gaussian metric only uses sqrt(y)).  When `bad` is not
// NULL, *bad |= 1 if any entry is negative, infinite or NaN (the caller zeroes it first);
// y_perm == NULL only checks.
cudaError_t permute_measurements(int LS, int LE, const float* y, float* y_perm, int K, int take_sqrt, int blocks,
                                 cudaStream_t stream, unsigned* bad);

// Record the thread-local message that ptylm_last_error() returns (shared by all entry points).
void set_last_error(const char* msg);

// Read-only view of a single-problem context for the learned initialisation: measurements
// in team-register order (sqrt(y) for the Gaussian metric), positions, twiddles, sizes.
struct CtxView {
    const float* y_team;
    const int2* pos;
    const float2* tw;
    int K, ny, nx, m, loss, num_sms;
    cudaStream_t stream;
};
bool ctx_view(const struct ptylm_ctx* c, CtxView* v);

// Launch kernel `kid` for the tile (2^LS side, 2^LE values per thread) on `grid` CTAs.
cudaError_t kernel_launch(int LS, int LE, int kid, const PtyArgs& a, int grid, cudaStream_t stream);

}  // namespace ptylm
