// Shared pieces of the batched kernels (forward propagation and adjoint): launch
// arguments, the bounded grid barrier, trajectory grouping and the register-tiled complex
// matrix product through shared memory.
#pragma once

#include "common.cuh"
#include "stage.cuh"

namespace tdagw {
namespace batched {

constexpr int kBThreads = 512;
constexpr int kTileB = 32;      // trajectories per CTA block (max)
constexpr int kChunk = 16;      // reduction-dimension chunk staged in shared memory
constexpr int kLdA = 258;       // padded row of the staged A chunk (float2), 16-B aligned

struct BatchArgs {
    // factors / kernel
    const float2* U;      // N x ldu
    const float2* V;      // N x ldu
    const float* S;       // r
    const float2* diag;   // N
    const float2* K;      // N x N (dense mode)
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
};

__device__ __forceinline__ uint64_t gtimer_b() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acq(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_rel(unsigned long long* p) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

// grid barrier with a monotonic arrival counter (see lr_persistent.cu); all threads call
static __device__ bool bgrid_sync(const BatchArgs& a, unsigned& gen, int* abort_s) {
    __syncthreads();
    if (threadIdx.x == 0 && !*abort_s) {
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x;
        red_rel(a.bar);
        const uint64_t t0 = gtimer_b();
        while (ld_acq(a.bar) < target) {
            if (gtimer_b() - t0 > a.wait_ns || *(volatile int*)a.err) {
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
// A[m lda + q] (NN: A is M x Q, rows m).  Bm rows q at Bm + q ldb.  Output accumulated in
// registers: thread (ty, tx) owns rows m = 4 ty + {0..3} (+ 256 per pass) and columns
// b = 4 tx + {0..3}; 64 x 8 threads cover 256 x 32 outputs per pass.
template <bool TRANS>
static __device__ void block_gemm(const float2* __restrict__ A, int64_t lda, int M, int Q,
                           const float2* __restrict__ Bm, int64_t ldb, int nb,
                           float2* __restrict__ out, int64_t ldo, bool accumulate_diag,
                           const float2* __restrict__ diag, const float2* __restrict__ xd,
                           float2* sA, float2* sB) {
    const int tid = threadIdx.x;
    const int tx = tid % 8, ty = tid / 8;  // 8 column groups of 4, 64 row groups of 4
    for (int m0 = 0; m0 < M; m0 += 256) {
        float2 c[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) c[u][v] = make_float2(0.f, 0.f);
        const int mrows = min(256, M - m0);
        for (int q0 = 0; q0 < Q; q0 += kChunk) {
            const int qn = min(kChunk, Q - q0);
            // stage A chunk as sA[q][m] (kChunk x 256, padded rows) and B chunk as
            // sB[q][b] (kChunk x 32); global reads run along contiguous memory
            for (int e = tid; e < kChunk * 256; e += kBThreads) {
                int q, m;
                if (TRANS) {  // A rows are q: consecutive threads read consecutive m
                    q = e / 256;
                    m = e % 256;
                } else {      // A rows are m: consecutive threads read consecutive q
                    m = e / kChunk;
                    q = e % kChunk;
                }
                float2 v = make_float2(0.f, 0.f);
                if (q < qn && m < mrows) {
                    if (TRANS) {
                        v = __ldcg(A + (int64_t)(q0 + q) * lda + m0 + m);
                        v.y = -v.y;
                    } else {
                        v = __ldcg(A + (int64_t)(m0 + m) * lda + q0 + q);
                    }
                }
                sA[q * kLdA + m] = v;
            }
            for (int e = tid; e < kChunk * kTileB; e += kBThreads) {
                const int q = e / kTileB, b = e % kTileB;
                sB[e] = (q < qn && b < nb) ? __ldcg(Bm + (int64_t)(q0 + q) * ldb + b) : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 4
            for (int q = 0; q < kChunk; ++q) {
                const float4 a01 = *reinterpret_cast<const float4*>(sA + q * kLdA + 4 * ty);
                const float4 a23 = *reinterpret_cast<const float4*>(sA + q * kLdA + 4 * ty + 2);
                const float4 b01 = *reinterpret_cast<const float4*>(sB + q * kTileB + 4 * tx);
                const float4 b23 = *reinterpret_cast<const float4*>(sB + q * kTileB + 4 * tx + 2);
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
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = m0 + 4 * ty + u;
            if (m >= M) continue;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int b = 4 * tx + v;
                if (b >= nb) continue;
                float2 r = c[u][v];
                if (accumulate_diag) r = cfma(diag[m], __ldcg(xd + (int64_t)m * ldb + b), r);
                out[(int64_t)m * ldo + b] = r;
            }
        }
    }
}


}  // namespace batched
}  // namespace tdagw
