// Shared pieces of the batched kernels (forward propagation and adjoint): launch
// arguments, the bounded grid barrier, trajectory grouping and the register-tiled complex
// matrix product through shared memory.
#pragma once

#include "common.cuh"
#include "persist.cuh"
#include "stage.cuh"

namespace tdagw {
namespace batched {

constexpr int kBThreads = 512;
constexpr int kTileB = 32;      // trajectories per CTA block (max)
constexpr int kChunk = 16;      // reduction-dimension chunk staged in shared memory
constexpr int kLdA = 272;       // staged A chunk row (float2): 256 columns + room for the
                                // padded per-slice layouts of a split reduction
constexpr int kKSplitMax = 4;   // reduction-dimension split of block_gemm for small M
// shared memory of block_gemm (float2): staged A chunk, then one B chunk per slice
constexpr int kGemmSmem = kChunk * kLdA + kKSplitMax * kChunk * kTileB;

struct BatchArgs {
    // factors / kernel
    const float2* U;      // N x ldu
    const float2* V;      // N x ldu
    const float* S;       // r
    const float2* diag;   // N
    const float2* kblk;   // k-block reading of K^diag (Nk x P x P, (k P + p) P + q) or nullptr
    const float2* K;      // N x N (dense mode)
    // channel-wise mode (Eq. svd-channel-wise): V and U segments, the layout, and the P x P
    // tables uoff [p P + q], voff [q P + p], z [p P + q] (S, P, Y then span m->stot columns)
    const float2* Vch;
    const float2* Uch;
    const ChMeta* chm;
    const int* choff;
    // model (per pair element)
    const float2* dx;
    const float2* dy;
    const float2* vx;
    const float2* gap;
    // batched state, N x Bp row-major (column b = trajectory b in sorted order)
    float2* X;
    float2* Ssum;
    float2* Ccomp;
    float2* acc;
    float2* dS;
    // low-rank intermediates
    float2* P;            // Rg x r x Bp
    float2* Y;            // r x Bp
    // per trajectory (sorted order)
    const double* Etab;   // B x ldE
    const float2* dir;    // B (dir_x, dir_y)
    const int* act;       // T_max: active trajectories during step n
    double* red;          // Rg x Bp x 3 observables partials
    double* obs;          // (T_max + 1) x B x 3 (sorted order)
    unsigned long long* bar;
    int* err;
    int64_t N, ldE;
    int Nk, Nb, r, ldu, Bp, B, Tmax, Rg, Tg, mode, kahan, c1;
    float occ[4];
    float dt;
    unsigned long long wait_ns;
    // adjoint support: global step offset of this launch, checkpoints of the compensated
    // state every ck_period steps, and per-stage records of (X_s, dSigma_s) for the steps
    // of this launch (layout [step * 4 + stage][N][Bp])
    int n0, ck_period;
    float2* ckS;
    float2* ckC;
    float2* recX;
    float2* recDS;
    int extra_arrivals;  // > 0 only for the timeout test: the grid barrier can never complete
};

// grid barrier with a monotonic arrival counter (see persist::grid_sync); all threads call
static __device__ bool bgrid_sync(const BatchArgs& a, unsigned& gen, int* abort_s) {
    __syncthreads();
    if (threadIdx.x == 0 && !*abort_s) {
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x + a.extra_arrivals;
        persist::red_release_add64(a.bar, 1ull);
        const uint64_t t0 = persist::gtimer();
        while (persist::ld_acquire64(a.bar) < target) {
            if (persist::gtimer() - t0 > a.wait_ns || *(volatile int*)a.err) {
                atomicExch(a.err, 1);
                *abort_s = 1;
                break;
            }
            __nanosleep(32);
        }
        gen += 1;
    }
    __syncthreads();
    return !*(volatile int*)abort_s;
}

// trajectories [b0, b1) of group tg among the B_act active ones
__device__ __forceinline__ void group_range(int Bact, int Tg, int tg, int& b0, int& b1) {
    b0 = (int)((int64_t)tg * Bact / Tg);
    b1 = (int)((int64_t)(tg + 1) * Bact / Tg);
}

// C[m][b] (+)= sum_q opA(q, m) Bm[q][b] for m in [0, M), b in [0, nb) (nb <= 32),
// q in [0, Q).  opA(q, m) = conj(A[q lda + m]) (TRANS: A is Q x M, rows q) or
// A[m lda + q] (NN: A is M x Q, rows m).  Bm rows q at Bm + q ldb.  Outputs accumulate in
// registers, 4 x 4 complex per thread (8 column groups x row groups).  For small M (a
// CTA's few rows) the reduction dimension is split over ks = 2 or 4 thread slices, each
// covering 256 / ks rows with its own staged chunk; the slices' partial tiles are added in
// fixed slice order through the (then idle) staging memory, so results are deterministic.
// sA: kChunk x kLdA float2 followed by sB: kKSplitMax x kChunk x kTileB float2 (contiguous).
template <bool TRANS, int LKS, bool ACC>
static __device__ void block_gemm_split(const float2* __restrict__ A, int64_t lda, int M, int Q,
                           const float2* __restrict__ Bm, int64_t ldb, int nb,
                           float2* __restrict__ out, int64_t ldo, bool accumulate_diag,
                           const float2* __restrict__ diag, const float2* __restrict__ xd,
                           float2* sA, float2* sB) {
    const int tid = threadIdx.x;
    constexpr int lks = LKS;                   // log2 of the split (compile time: constant
    constexpr int ks = 1 << lks;               // shared-memory offsets in the inner loop)
    constexpr int lmt = 8 - lks;               // log2 of the rows per pass
    constexpr int Mt = 1 << lmt;
    constexpr int ng = kBThreads >> lks;       // threads per slice
    const int slice = tid / ng, tl = tid % ng;
    const int tx = tl % 8, ty = tl / 8;        // 8 column groups of 4, 64 / ks row groups of 4
    constexpr int lds = Mt + 2;                // staged row of one slice (even: float4 reads)
    float2* sAs = sA + slice * kChunk * lds;
    float2* sBs = sB + slice * kChunk * kTileB;
    for (int m0 = 0; m0 < M; m0 += Mt) {
        float2 c[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) c[u][v] = make_float2(0.f, 0.f);
        const int mrows = min(Mt, M - m0);
        for (int q0 = 0; q0 < Q; q0 += ks * kChunk) {
            // stage ks chunks (slice s: q in [q0 + s kChunk, q0 + (s + 1) kChunk)); global
            // reads run along contiguous memory
            for (int e = tid; e < kChunk * 256; e += kBThreads) {
                const int s = e >> (lmt + 4), e2 = e & ((kChunk << lmt) - 1);
                int q, m;
                if (TRANS) {  // A rows are q: consecutive threads read consecutive m
                    q = e2 >> lmt;
                    m = e2 & (Mt - 1);
                } else {      // A rows are m: consecutive threads read consecutive q
                    m = e2 >> 4;
                    q = e2 & (kChunk - 1);
                }
                const int qg = q0 + s * kChunk + q;
                float2 v = make_float2(0.f, 0.f);
                if (qg < Q && m < mrows) {
                    if (TRANS) {
                        v = __ldcg(A + (int64_t)qg * lda + m0 + m);
                        v.y = -v.y;
                    } else {
                        v = __ldcg(A + (int64_t)(m0 + m) * lda + qg);
                    }
                }
                sA[(s * kChunk + q) * lds + m] = v;
            }
            for (int e = tid; e < (kChunk * kTileB << lks); e += kBThreads) {
                const int s = e / (kChunk * kTileB), q = (e / kTileB) % kChunk, b = e % kTileB;
                const int qg = q0 + s * kChunk + q;
                sB[e] = (qg < Q && b < nb) ? __ldcg(Bm + (int64_t)qg * ldb + b) : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 4
            for (int q = 0; q < kChunk; ++q) {
                const float4 a01 = *reinterpret_cast<const float4*>(sAs + q * lds + 4 * ty);
                const float4 a23 = *reinterpret_cast<const float4*>(sAs + q * lds + 4 * ty + 2);
                const float4 b01 = *reinterpret_cast<const float4*>(sBs + q * kTileB + 4 * tx);
                const float4 b23 = *reinterpret_cast<const float4*>(sBs + q * kTileB + 4 * tx + 2);
                const float2 av[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                                      make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
                const float2 bv[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                                      make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) c[u][v] = cfma(av[u], bv[v], c[u][v]);
            }
            __syncthreads();
        }
        if (ks > 1) {
            // partial tiles of slices 1..ks-1 -> staging memory; slice 0 adds them in order
            float2* red = sA;
            if (slice > 0)
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        red[((slice - 1) * Mt + 4 * ty + u) * kTileB + 4 * tx + v] = c[u][v];
            __syncthreads();
            if (slice == 0)
                for (int s = 1; s < ks; ++s)
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            c[u][v] = cadd(c[u][v], red[((s - 1) * Mt + 4 * ty + u) * kTileB + 4 * tx + v]);
        }
        if (slice == 0)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int m = m0 + 4 * ty + u;
                if (4 * ty + u >= mrows) continue;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int b = 4 * tx + v;
                    if (b >= nb) continue;
                    float2 r = c[u][v];
                    if (accumulate_diag) r = cfma(diag[m], __ldcg(xd + (int64_t)m * ldb + b), r);
                    if (ACC) r = cadd(r, out[(int64_t)m * ldo + b]);
                    out[(int64_t)m * ldo + b] = r;
                }
            }
        if (ks > 1) __syncthreads();  // staging memory is reused by the next pass
    }
}

// k-block reading of K^diag: out[row][b] += sum_q B_k[p][q] x[k P + q][b] (CT: the conjugate
// transpose, conj(B_k[q][p]), for K^H) for rows [ra, ra + nrows) (whole k-points) and columns
// [b0, b0 + nb); row = k P + p, B_k[p][q] at kblk[(k P + p) P + q].
template <int NB, bool CT>
static __device__ void kblock_term(const float2* __restrict__ kblk, const float2* __restrict__ x,
                                   float2* __restrict__ out, int64_t ld, int64_t ra, int nrows, int b0, int nb) {
    constexpr int P = NB * NB;
    for (int e = threadIdx.x; e < nrows * nb; e += kBThreads) {
        const int64_t row = ra + e / nb;
        const int b = b0 + e % nb;
        const int64_t k0 = row - row % P;
        const int p = (int)(row % P);
        float2 s = __ldcg(out + row * ld + b);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const float2 bq = CT ? cconj(kblk[(k0 + q) * P + p]) : kblk[row * P + q];
            s = cfma(bq, __ldcg(x + (k0 + q) * ld + b), s);
        }
        out[row * ld + b] = s;
    }
}

// ACC: add the product to out instead of overwriting it
template <bool TRANS, bool ACC = false>
static __device__ void block_gemm(const float2* __restrict__ A, int64_t lda, int M, int Q,
                           const float2* __restrict__ Bm, int64_t ldb, int nb,
                           float2* __restrict__ out, int64_t ldo, bool accumulate_diag,
                           const float2* __restrict__ diag, const float2* __restrict__ xd,
                           float2* sA, float2* sB) {
    static_assert(kKSplitMax == 4, "split variants below");
    if (4 * M <= 256)
        block_gemm_split<TRANS, 2, ACC>(A, lda, M, Q, Bm, ldb, nb, out, ldo, accumulate_diag, diag, xd, sA, sB);
    else if (2 * M <= 256)
        block_gemm_split<TRANS, 1, ACC>(A, lda, M, Q, Bm, ldb, nb, out, ldo, accumulate_diag, diag, xd, sA, sB);
    else
        block_gemm_split<TRANS, 0, ACC>(A, lda, M, Q, Bm, ldb, nb, out, ldo, accumulate_diag, diag, xd, sA, sB);
}


}  // namespace batched
}  // namespace tdagw
