// batch.h -- device-side description of a batch of independent reconstructions and the
// launchers of the persistent per-position kernels that serve all of them in one launch.
#pragma once
#include <cuda_runtime.h>

namespace ptylm {

// One object-only problem of the batch (Sec. 2, Eq. cdp): its scan, measurements, probe,
// frequency cache and where its object lives inside the concatenated batch vectors.
struct BatchProblem {
    const int2* pos;     // [K] (row, column) of each patch
    const float* y;      // [K][M] measurements in team-register order (sqrt(y) for Gaussian)
    float2* a_cache;     // [K][M] cache a = psihat (d2l)^(1/2) / zeta of the last linearisation
    float* trp;          // [K][T] per-thread sums of d2l of the last linearisation (T = M / E)
    const float2* P;     // [M] probe
    long z_off;          // first element of this problem's object in the batch vectors
    int K, nx, LS, loss;
    float b;             // background b (+ the surrogate s_t inside the batched LM)
    int LE;              // log2 of the values per thread of its FFT tile (5, or 4 for S <= 64)
};

// A work item: positions k0 + team + teams * j (j < per_team) of problem `prob`, where
// teams = 512 / (S^2 / E) is the number of thread teams a 512-thread CTA holds for the
// problem's probe side S and values per thread E (16, 4 and 1 for S = 32, 64, 128 with
// E = 32; 8 and 2 for S = 32, 64 with E = 16).
struct BatchItem {
    int prob, k0, per_team, pad;
};

struct BatchArgs {
    const BatchProblem* probs;
    const BatchItem* items;
    int n_items;
    unsigned* work;       // next item to take (0 on entry, restored to 0 on exit)
    unsigned* done;       // CTAs finished (0 on entry, restored to 0 on exit)
    const float2* tw;     // twiddles W_S^j for S = 32, 64, 128, concatenated (224 entries)
    const float2* V;      // input batch vector: objects (forward) or directions (matvec)
    float2* out;          // output batch vector, accumulated into (gradient / GGN product)
    double* f;            // [B][2]: error metric and ||grad_zeta l||^2 per problem (forward)
    const int* active;    // [B] or NULL: items of problems with active[b] == 0 are skipped
};

constexpr int BATCH_THREADS = 512;
constexpr int BATCH_TW = 32 + 64 + 128;

enum BatchKernel { BK_FWD_LOSS = 0, BK_FWD_CACHE = 1, BK_MATVEC = 2, BK_COUNT = 3 };

// Opt in to the kernels' shared memory and return how many CTAs of each fit on one SM.
cudaError_t batch_prepare(int* ctas_per_sm);
cudaError_t batch_launch(int kernel, const BatchArgs& a, int grid, cudaStream_t stream);
// Closed-form diagonal of every problem's GGN in real coordinates at its linearisation point
// (App. B; the single-problem k_diag_object): D[z_off + n] += sum over the positions k of
// problem b whose patch holds n of |P[n - r_k]|^2 tr_k / (2M), tr_k = sum of trp[k][.],
// for the problems with mask[b] != 0 (D zeroed there beforehand).  pos_first: [B + 1]
// prefix sums of the position counts; one block per position of the whole batch.
cudaError_t batch_diag_launch(const BatchProblem* probs, const int* pos_first, int B, int total_positions,
                              const int* mask, float* D, cudaStream_t stream);

// Measurements of K positions of side 2^LS from the team-register order of the tile with
// 2^le_from values per thread to that with 2^le_to (le in {4, 5}, LS in {5, 6}); src and
// dst must not overlap.
cudaError_t batch_relayout_measurements(int LS, int le_from, int le_to, const float* src, float* dst, int K, int blocks,
                                        cudaStream_t stream);

}  // namespace ptylm
