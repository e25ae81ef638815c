// Batched low-rank TD-aGW propagation on the fifth-generation tensor cores, with the
// truncated-SVD factors of Eq. svd_acc stored as split FP16 pairs (hi + lo, 8 bytes per
// complex element like complex64).
//
// Per RK4 stage the two products of the low-rank contraction,
//   Y = V^H X  (r x B)   and   dSigma = K^diag o X + U (S o Y)  (N x B),
// run as real tcgen05 kind::f16 MMAs with FP32 accumulation in tensor memory.  Shape: the
// small operand (a group of up to 64 trajectories, expanded to 128 real rows) is the MMA's
// A operand and lives in tensor memory, the factor (the large, streamed operand) is the
// B operand, 256 rows per tile, read from shared memory: M = 128, N = 256, K = 16.  Keeping
// A out of shared memory halves the operand traffic of the shared memory per MMA, which
// bounds the MMA rate when both operands are read from it.  Complex arithmetic: the factor
// is read as an interleaved real matrix (re, im per complex column) and each trajectory's
// value becomes two real rows, so one real product yields the real and imaginary parts in
// adjacent accumulator lanes.  Split FP16: with a = s (a_hi + a_lo), each product is
// accumulated as a_hi b_hi + a_lo b_hi + a_hi b_lo (three MMAs; the dropped a_lo b_lo is
// 2^-22 relative).  Power-of-two scales keep the FP16 values in range: 2^(13 - e) with 2^e
// above the largest magnitude, for U and V (measured once when the tiles are made) and,
// per trajectory, for X (the exact maximum of the stage input) and for S o Y (bound
// max|S| max_j ||v_j|| sqrt(2N) max|X|).
//
// Work of one stage (one cooperative launch for the whole propagation, one CTA per SM):
//   A  partials of V^H X over K-ranges of rows: CTA items (trajectory group, 256-row tile
//      of V^H, K-range).  The V^H tiles (pre-tiled 32 KB blocks in the MMA's shared-memory
//      layout) stream through a ring by bulk copies; the worker warps write the expanded
//      split X block of every chunk straight into tensor memory.
//   -- grid barrier --
//   B  S o (sum of the partials, fixed order), scaled for FP16.
//   -- grid barrier --
//   C  items (256-row tile of U, trajectory group): the U tiles stream through the ring,
//      the workers write the expanded split S o Y blocks into tensor memory; the
//      accumulator (128 lanes x 256 rows) is staged through shared memory in quarters and
//      the commutator + RK4 epilogue (Eq. tdagw) runs per (k, b) block; each item then
//      counts its row tile (release), and the next stage's phase A items wait only for
//      the tiles of their K-ranges instead of a grid barrier.
// The channel-wise mode (Eq. svd-channel-wise, a second instantiation) runs phase A per V
// segment and phase C per U segment (low-rank columns and the dense diagonal channel of an
// output pair) with gathered operand rows, writes dSigma to global memory, and runs the
// epilogue as a fourth phase by 64-row quarters, with grid barriers between all phases.
// Roles: warp 0 streams the factor tiles into the ring (it only reads static tiles, so it
// stays out of the grid barriers and keeps copies in flight across them), warp 1 issues
// the MMAs, warps 2-9 build the tensor-memory operands and drain the accumulator.  Every
// wait is bounded; on expiry the kernel records an error, lets its own copies and MMAs
// finish (bounded waits), frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "batched_common.cuh"
#include "persist.cuh"
#include "tc_ptx.cuh"

namespace tdagw {

namespace {

using namespace batched;
using namespace persist;

constexpr int kWorkers = 256;
constexpr int kTcThreads = kWorkers + 64;  // warp 0: copies, warp 1: MMAs, warps 2-9: workers
constexpr int kSyncThreads = kWorkers + 32;  // grid-barrier participants: MMA warp + workers
#ifndef TDAGW_TC_RING
#define TDAGW_TC_RING 4
#endif
constexpr int kRing = TDAGW_TC_RING;       // ring slots of one factor tile each
#ifndef TDAGW_TC_ABUF
#define TDAGW_TC_ABUF 4
#endif
constexpr int kAbuf = TDAGW_TC_ABUF;       // small-operand blocks in tensor memory
constexpr int kCmb = 16;                   // chunk-completion barriers; every wait on one
                                           // targets a chunk < kCmb chunks behind the
                                           // waiter's next chunk, so parities cannot alias
constexpr int kRows = 256;                 // factor rows per tile: the MMA's N
constexpr uint32_t kTile = 32768;          // 256 rows x 32 real columns, hi (16 KB) + lo (16 KB)
constexpr uint32_t kHalf = 16384;
constexpr int kKc = 32;                    // real reduction columns per tile (16 complex)
constexpr int kGroup = 64;                 // trajectories per group: the MMA's M = 2 x 64
constexpr uint32_t kLbo = 128, kSbo = (kKc / 8) * 128;
constexpr uint32_t kStg = 32768;           // staged quarter tile: 64 rows x 64 trajectories
constexpr int kTmemCols = 512;
constexpr uint32_t kAcol = 256;            // tensor-memory columns of the operand blocks
// The workers read the values of each operand block (16 rows of X or of S o Y for their
// trajectories) through shared memory: asynchronous copies issued kSrcAhead chunks ahead
// into kSrcSlots slots of 8 KB (the staging buffer of the epilogue, idle while the
// operands stream), so the block builds do not wait on L2 latency.
constexpr int kSrcSlots = 4, kSrcAhead = 3;
static_assert(kSrcSlots * 8192 <= (int)32768 && kSrcAhead < kSrcSlots, "operand source slots");
static_assert(kRing >= 2 && kRing < kCmb, "ring depth");
static_assert(kAcol + 32 * kAbuf <= (uint32_t)kTmemCols, "tensor memory");
#ifndef TDAGW_TC_EVICT_FIRST
#define TDAGW_TC_EVICT_FIRST 1  // factor tiles are streamed with an L2 evict-first policy
#endif

// staged quarter tile: 64 rows x 64 trajectories of float2, columns XOR-swizzled by row so
// that both the row-wise writes and the trajectory-wise reads avoid bank conflicts
__device__ __forceinline__ int ds_index(int row, int bl) {
    return row * 64 + (bl ^ (row & 31));
}

struct TcArgs {
    const unsigned char* tU;  // Nt x nchU tiles of U (256 rows) x 32 real columns
    const unsigned char* tV;  // Mt x nchV tiles of V^T (256 rows j) x 32 real columns (16 rows i)
    float2* Ys;               // rp x Bp: S o Y scaled for FP16 (phase B)
    float2* P;                // KS x rp x Bp raw partials of V^H X
    unsigned* xmax;           // 3 x Bp: max(|Re|, |Im|) of the stage input (float bits)
    const float* S;
    const float2* diag;
    const float2* dx;
    const float2* dy;
    const float2* vx;
    const float2* gap;
    float2* X;
    float2* Ssum;
    float2* Ccomp;
    float2* acc;
    const double* Etab;
    const float2* dir;
    const int* act;
    double* red;  // Nt x Bp x 3 (per phase C row-tile item)
    double* obs;  // (Tmax + 1) x B x 3
    unsigned long long* bar;
    int* err;
    int64_t N, ldE;
    int Nk, r, rp, Nt, Mt, nchU, nchV, Bp, B, Tmax, kahan, c1;
    int gc_max;     // phase C trajectory groups at most (1 .. B / 8); 0: fill the CTAs
    int ks_max;     // phase A K-ranges at most; 0: fill the CTAs
    // adjoint support: global step of this launch's first step, checkpoints of the
    // compensated state every ck_period steps, per-stage records of (X_s, dSigma_s) for the
    // steps of this launch ([step * 4 + stage][N][Bp]); null pointers: off
    int n0, ck_period;
    float2* ckS;
    float2* ckC;
    float2* recX;
    float2* recDS;
    float occ[4];
    float dt;
    float su, sv;   // power-of-two scales of the U and V tiles
    float ybound;   // max|S| max_j ||v_j|| sqrt(2N): |(S o Y)_jb| <= ybound max|X_b|
    unsigned long long wait_ns;
    int Nred;       // tiles of the per-tile observable sums (red): row tiles, or quarters
    int extra_arrivals;  // > 0 only for the timeout test: the grid barrier can never complete
    // low-rank mode: per 256-row tile, the epilogue items completed so far (monotonic) and
    // max(|Re|, |Im|) of the new stage input per trajectory (float bits): a phase A item
    // waits only for the tiles of its K-range instead of a grid barrier
    unsigned long long* tdone;
    unsigned* xtile;
    int use_flags;  // low-rank mode: 1 the per-tile counters, 0 a grid barrier after the epilogue
    // Channel-wise mode (Eq. svd-channel-wise; a separate instantiation).  Phase A runs
    // over the V segments (segment q: its Mt_q 256-column tiles, mtq0[q] the first of them
    // in the padded column order, K over the Nk k-points in nchV chunks), phase C over the
    // U segments (segment p = [U^pq of the channels out of p | K^pp]: NtK 256-row tiles of
    // k-points, nchw[p] chunks of its columns), with the operand z_p = [S o y of those
    // channels (padded rows gpad) ; x_p]; phase C writes dSigma to dS (one partial slot per
    // K-range) and a fourth phase runs the commutator + RK4 epilogue by 64-row quarters of
    // the nte 256-row tiles of all N rows.
    const int* gpad;
    float2* dS;
    int npair, NtK, nte;
    int kcu;        // K-ranges of a U segment tile (partial dSigma slots dS + kc N Bp)
    float zbound;   // |z_p| <= zbound max|X_b|
    long long tvoff[kMaxPairs], tuoff[kMaxPairs];
    int mtq0[kMaxPairs + 1], ldvq[kMaxPairs], sbq[kMaxPairs], nlrq[kMaxPairs], gbq[kMaxPairs], nchw[kMaxPairs];
};

// Optional phase timestamps (build with -DTDAGW_TRACE): one thread per CTA records
// %globaltimer at the phase boundaries of stages kTraceFirst .. kTraceFirst + kTraceStages - 1
// (points 0-6: stage start, end of A items, after barrier 1, end of B, after barrier 2, end
// of C items, after barrier 3; 7: MMA thread done with C items; 8: producer done with C
// tiles), and per-role wait totals.
#ifdef TDAGW_TRACE
constexpr int kTraceFirst = 40, kTraceStages = 16;
__device__ unsigned long long g_trace_tc[160 * kTraceStages * 9];
#define TC_TRACE(who, k)                                                                         \
    do {                                                                                         \
        const int ts_ = tr_gs - kTraceFirst;                                                     \
        if ((who) && blockIdx.x < 160 && ts_ >= 0 && ts_ < kTraceStages)                         \
            g_trace_tc[(blockIdx.x * kTraceStages + ts_) * 9 + (k)] = gtimer();                   \
    } while (0)
// wait/issue time accumulators per CTA and traced stage: [0] MMA thread waiting for tiles,
// [1] for operand blocks, [2] for the accumulator, [3] issuing MMAs and commits, [4] copy
// thread waiting for a free slot, [5] issuing copies; worker 0: [6] waiting for a free
// operand block, [7] waiting for its source values, [8] storing to tensor memory
__device__ unsigned long long g_trace_w[160 * kTraceStages * 9];
#define TC_W_BEGIN(id) const uint64_t tw_##id = gtimer()
#define TC_W_END(id, k)                                                                          \
    do {                                                                                         \
        const int ts_ = tr_gs - kTraceFirst;                                                     \
        if (blockIdx.x < 160 && ts_ >= 0 && ts_ < kTraceStages)                                  \
            g_trace_w[(blockIdx.x * kTraceStages + ts_) * 9 + (k)] += gtimer() - tw_##id;         \
    } while (0)
#else
#define TC_TRACE(who, k) \
    do {                 \
    } while (0)
#define TC_W_BEGIN(id) \
    do {               \
    } while (0)
#define TC_W_END(id, k) \
    do {                \
    } while (0)
#endif

// bounded wait for the phase of the given parity (polling); false on expiry or abort
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, volatile int* abort_s,
                                        unsigned long long budget) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(b, parity)) return true;
        if ((i & 63) == 0) {
            if (abort_s && *abort_s) return false;
            if (gtimer() - t0 > budget) return false;
        }
    }
}
__device__ __forceinline__ void workers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory");
}
__device__ __forceinline__ void participants_sync() {
    asm volatile("bar.sync 2, %0;" ::"n"(kSyncThreads) : "memory");
}

// 2^(13 - e) for bound < 2^e (1 for a zero bound)
__device__ __forceinline__ float pow2_scale(float bound) {
    if (!(bound > 0.f)) return 1.f;
    int e;
    frexpf(bound, &e);
    e = max(e, -100);
    return ldexpf(1.f, 13 - e);
}
__device__ __forceinline__ void split16(float v, __half& hi, __half& lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}
__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// 8-byte asynchronous copy global -> shared (zero-filled when src_bytes is 0) and its
// per-thread completion groups
__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// grid barrier over the monotonic arrival counter among the MMA warp and the workers (the
// copy warp never waits on other CTAs)
__device__ bool tc_grid_sync(const TcArgs& a, unsigned& gen, int* abort_s) {
    participants_sync();
    if (threadIdx.x == 64 && !*abort_s) {
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x + a.extra_arrivals;
        red_release_add64(a.bar, 1ull);
        const uint64_t t0 = gtimer();
        while (ld_acquire64(a.bar) < target) {
            if (gtimer() - t0 > a.wait_ns || *(volatile int*)a.err) {
                atomicExch(a.err, 1);
                *abort_s = 1;
                break;
            }
            __nanosleep(32);
        }
    }
    gen += 1;
    participants_sync();
    return !*(volatile int*)abort_s;
}

// the three split products of one chunk: D (128 x 256) += A[tmem] (128 x 32) . F^T with F
// the 256 x 32 factor tile (two K = 16 steps each)
__device__ __forceinline__ void mma_chunk(uint32_t d, uint32_t a_tm, uint32_t f_addr, uint32_t idesc, bool first) {
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        const uint64_t fh = tc::sdesc(f_addr + ks * 256, kLbo, kSbo);
        const uint64_t fl = tc::sdesc(f_addr + kHalf + ks * 256, kLbo, kSbo);
        tc::mma_f16_ts(d, a_tm + ks * 8, fh, idesc, (first && ks == 0) ? 0u : 1u);
        tc::mma_f16_ts(d, a_tm + 16 + ks * 8, fh, idesc, 1u);
        tc::mma_f16_ts(d, a_tm + ks * 8, fl, idesc, 1u);
    }
}

// Observable sums of the epilogue in double-float (DF, FP32 pipes; FP64 arithmetic is
// slow on this GPU), widened to FP64 once per thread.
struct DF3 {
    DF p, j, o;
};

// Commutator + RK4 stage update of one (k, trajectory) block (Eq. tdagw; the arithmetic of
// the FP32 batched path), with the low-rank part of dSigma read from the staged quarter
// tile (block rows row0 .. row0 + NB^2 - 1, trajectory column bl) and K^diag o X added here.
// xm: running max(|Re|, |Im|) of the values written to X (the next stage input); ob: the
// thread's running sums of the observables (last stage).
template <int NB>
__device__ void stage_kb_tc(const TcArgs& a, int k, int b, int st, float E, float2 dr,
                            const float2* sDS, int row0, int bl, float& xm, DF3& ob, int64_t rec) {
    constexpr int NB2 = NB * NB;
    const int64_t Bp = a.Bp;
    float2 X[NB2], M[NB2];
#pragma unroll
    for (int g = 0; g < NB2; ++g) {
        const int64_t i = (int64_t)k * NB2 + g;
        X[g] = __ldcg(a.X + i * Bp + b);
        const float2 d1 = a.dx[i], d2 = a.dy[i];
        const float2 ds = cfma(a.diag[i], X[g], sDS[ds_index(row0 + g, bl)]);
        if (rec >= 0) {  // stage input and dSigma, for the adjoint's backward sweep
            a.recX[rec + i * Bp + b] = X[g];
            a.recDS[rec + i * Bp + b] = ds;
        }
        M[g] = make_float2(ds.x + E * (dr.x * d1.x + dr.y * d2.x), ds.y + E * (dr.x * d1.y + dr.y * d2.y));
    }
    // state loads of RB rows at a time, issued before any store of those rows (all rows
    // for two bands, one row for four: register budget)
    constexpr int RB = NB == 2 ? 2 : 1;
#pragma unroll
    for (int n0 = 0; n0 < NB; n0 += RB) {
        float2 XS[RB * NB], XC[RB * NB], AC[RB * NB];
#pragma unroll
        for (int q = 0; q < RB * NB; ++q) {
            const int64_t e = ((int64_t)k * NB2 + n0 * NB + q) * Bp + b;
            XS[q] = __ldcg(a.Ssum + e);
            XC[q] = __ldcg(a.Ccomp + e);
            AC[q] = st > 0 ? __ldcg(a.acc + e) : make_float2(0.f, 0.f);
        }
#pragma unroll
    for (int n = n0; n < n0 + RB; ++n)
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            const int g = n * NB + m;
            const int q = (n - n0) * NB + m;
            const int64_t i = (int64_t)k * NB2 + g;
            float2 comm = cscale(M[g], a.occ[m] - a.occ[n]);
#pragma unroll
            for (int l = 0; l < NB; ++l) {
                comm = cfma(M[n * NB + l], X[l * NB + m], comm);
                comm = csub(comm, cmul(X[n * NB + l], M[l * NB + m]));
            }
            const float2 h0 = gap_times(a.gap[i], X[g]);
            const float2 s = cadd(h0, comm);
            const float2 kv = make_float2(s.y, -s.x);
            const int64_t e = i * Bp + b;
            const float2 xs = XS[q], xc = XC[q];
            float2 Xn;
            if (st < 3) {
                const float2 ac = st == 0 ? kv : cadd(AC[q], cscale(kv, 2.f));
                a.acc[e] = ac;
                const float cn = st == 2 ? a.dt : 0.5f * a.dt;
                Xn = cadd(xs, cadd(xc, cscale(kv, cn)));
            } else {
                const float2 ac = cadd(AC[q], kv);
                const float2 inc = cscale(ac, a.dt / 6.f);
                float2 ns, nc;
                if (a.kahan) {
                    float ex, ey;
                    ns.x = two_sum(xs.x, inc.x, ex);
                    ns.y = two_sum(xs.y, inc.y, ey);
                    nc = make_float2(xc.x + ex, xc.y + ey);
                } else {
                    ns = cadd(xs, inc);
                    nc = xc;
                }
                a.Ssum[e] = ns;
                a.Ccomp[e] = nc;
                Xn = cadd(ns, nc);
                const float2 rho = (n == m) ? make_float2(Xn.x + a.occ[n], Xn.y) : Xn;
                const float2 d1 = a.dx[i], v1 = a.vx[i];
                ob.p.add_prod(rho.x, d1.x);
                ob.p.add_prod(rho.y, d1.y);
                ob.j.add_prod(rho.x, v1.x);
                ob.j.add_prod(rho.y, v1.y);
                if (n == m && n == a.c1) ob.o.add(rho.x);
            }
            a.X[e] = Xn;
            xm = fmaxf(xm, fmaxf(fabsf(Xn.x), fabsf(Xn.y)));
        }
    }
}

// Trajectory groups of phase C: at most kGroup trajectories each and, where the row tiles
// leave CTAs idle, more groups (>= 8 trajectories each, at most gc_max when set).
__host__ __device__ __forceinline__ int group_count(int Bact, int Nt, int nctas, int gc_max) {
    const int g_min = (Bact + kGroup - 1) / kGroup;
    int g_fill = min(max(1, nctas / Nt), (Bact + 7) / 8);
    if (gc_max > 0) g_fill = min(g_fill, gc_max);
    return max(g_min, g_fill);
}
struct Groups {
    int G, KS;  // phase A: trajectory groups, K-ranges
    int GC;     // phase C: trajectory groups
};
__device__ __forceinline__ Groups stage_groups(const TcArgs& a, int Bact) {
    Groups q;
    q.G = (Bact + kGroup - 1) / kGroup;
    q.GC = group_count(Bact, a.Nt, (int)gridDim.x, a.gc_max);
    int ks = (int)gridDim.x / max(1, q.G * a.Mt);
    if (a.ks_max > 0) ks = min(ks, a.ks_max);
    q.KS = max(1, min(ks, a.nchV));
    return q;
}
// phase A item -> (trajectory group, V^H tile, K-range and its chunks)
struct ItemA {
    int g, m, ks, c0, c1;
};
__device__ __forceinline__ ItemA item_a(const TcArgs& a, const Groups& q, int item) {
    ItemA it;
    it.g = item % q.G;
    it.m = (item / q.G) % a.Mt;
    it.ks = item / (q.G * a.Mt);
    it.c0 = (int)((int64_t)it.ks * a.nchV / q.KS);
    it.c1 = (int)((int64_t)(it.ks + 1) * a.nchV / q.KS);
    return it;
}

// Observables of step n from the Nred per-tile partial sums (channel-wise mode, where
// Nred is large): one warp per trajectory, the lanes take every 32nd tile and a butterfly
// sums the lanes, in a fixed order.  gw, nw: the calling warp and the number of warps.
__device__ void tc_obs_warp(const TcArgs& a, int n, int gw, int nw, int lane) {
    for (int b = gw; b < a.act[a.n0 + n - 1]; b += nw) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int t = lane; t < a.Nred; t += 32) {
            const double* rr = a.red + ((int64_t)t * a.Bp + b) * 3;
            s0 += __ldcg(rr);
            s1 += __ldcg(rr + 1);
            s2 += __ldcg(rr + 2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            double* o = a.obs + ((int64_t)n * a.B + b) * 3;
            o[0] = s0 / a.Nk;
            o[1] = s1 / a.Nk;
            o[2] = s2 / a.Nk;
        }
    }
}

// phase A tile index mt (padded column order) -> V segment q and its tile m (channel-wise)
__device__ __forceinline__ void seg_of_mt(const TcArgs& a, int mt, int& q, int& m) {
    q = 0;
    while (q + 1 < a.npair && a.mtq0[q + 1] <= mt) ++q;
    m = mt - a.mtq0[q];
}

template <int NB, bool CHT>
__global__ void __launch_bounds__(kTcThreads, 1) batched_tc_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ring = smem;
    float2* sDS = reinterpret_cast<float2*>(ring + kRing * kTile);
    // per-thread observable sums of an item: written after its last staged quarter is
    // consumed, read before the next item's operand sources are copied (they share memory)
    double* sred = reinterpret_cast<double*>(sDS);
    float* ssc = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sDS) + kStg);
    unsigned* smx = reinterpret_cast<unsigned*>(ssc + kGroup);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smx + kGroup);
    uint64_t* full = bars;
    uint64_t* cmb = full + kRing;     // MMAs of chunk q complete (one commit per chunk)
    uint64_t* afull = cmb + kCmb;     // operand block written (workers -> MMA)
    uint64_t* accf = afull + kAbuf;   // accumulator written (MMA -> workers)
    uint64_t* acce = accf + 1;        // accumulator drained (workers -> MMA)
    uint64_t* fin = acce + 1;         // last MMAs complete (teardown)
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = tid == 0, mma = tid == 32, worker = warp >= 2;
    const bool in_sync = warp >= 1;  // grid-barrier participants (lanes 1-31 of warp 0 idle)
    const int wt = tid - 64;  // worker index
    // worker warps: tensor-memory lane quarter (rows 32 q .. 32 q + 31 of the operand and of
    // the accumulator) and half (which columns of a block the warp writes or reads)
    const int wq = warp & 3, wh = (warp - 2) >> 2;
    const int orow = 32 * wq + lane;           // operand / accumulator row: 2 bl + comp
    const int obl = orow >> 1, ocomp = orow & 1;
    constexpr int NB2 = NB * NB;
    const unsigned long long budget = a.wait_ns;
    volatile int* vabort = &abort_s;
    // abort flag as one value per warp (lane 0's read): guards of the warp-collective
    // tensor-memory loads and stores must not diverge
    auto warp_abort = [&]() { return __shfl_sync(0xffffffffu, *vabort, 0) != 0; };

    if (tid == 0) {
        abort_s = 0;
        for (int s = 0; s < kRing; ++s) mbar_init(full + s, 1);
        for (int s = 0; s < kCmb; ++s) mbar_init(cmb + s, 1);
        for (int s = 0; s < kAbuf; ++s) mbar_init(afull + s, kWorkers / 32);
        mbar_init(accf, 1);
        mbar_init(acce, kWorkers);
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base, kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;

    uint32_t ppos = 0;  // producer: tiles issued so far (ring position)
    uint32_t mpos = 0;  // MMA thread: tiles consumed so far
    uint32_t bu = 0;    // uses of the operand blocks (MMA thread and workers)
    uint32_t acnt = 0;  // uses of the accumulator (MMA thread and workers)
    int gch = 0;        // chunks so far (all roles count the same sequence)
    int slot_ch[kRing]; // producer: chunk that last used each ring slot
    int buf_ch[kAbuf];  // workers: chunk that last used each operand block
    for (int q = 0; q < kRing; ++q) slot_ch[q] = -1;
    for (int q = 0; q < kAbuf; ++q) buf_ch[q] = -1;
    unsigned gen = 0;
    bool ok = true;
    unsigned long long tdone_target = 0;  // low-rank mode: epilogue items per tile so far
    int tr_gs = 0;  // stage of the phase timestamps (traced builds)
    (void)tr_gs;
    auto fail = [&]() {
        atomicExch(a.err, 1);
        abort_s = 1;
    };
    // wait until the MMAs of chunk q are complete (q < 0: nothing to wait for)
    auto chunk_done = [&](int q) -> bool {
        if (q < 0 || gch - q >= kCmb) return true;
        return mb_wait(cmb + q % kCmb, (uint32_t)(q / kCmb) & 1u, vabort, budget);
    };
    const uint64_t ef_policy = TDAGW_TC_EVICT_FIRST ? policy_evict_first() : 0ull;
    // producer: one factor tile (chunk gch) into the next ring slot
    auto issue = [&](const unsigned char* src) {
        if (*vabort) return;
        const uint32_t slot = ppos % kRing;
        if (!chunk_done(slot_ch[slot])) {
            fail();
            return;
        }
        slot_ch[slot] = gch;
        mbar_expect_tx(full + slot, kTile);
        if (TDAGW_TC_EVICT_FIRST)
            bulk_g2s_hint(ring + slot * kTile, src, kTile, full + slot, ef_policy);
        else
            bulk_g2s(ring + slot * kTile, src, kTile, full + slot);
        ++ppos;
    };
    // MMA thread: wait for the next tile; returns its shared-memory address (0 on failure)
    auto next_tile = [&]() -> uint32_t {
        const uint32_t slot = mpos % kRing, use = mpos / kRing;
        if (*vabort || !mb_wait(full + slot, use & 1u, vabort, budget)) {
            fail();
            return 0u;
        }
        ++mpos;
        return tc::smem_u32(ring + slot * kTile);
    };
    // MMA thread: one chunk (one factor tile and the operand block of the chunk)
    auto mma_step = [&](uint32_t idesc, bool first) {
        TC_W_BEGIN(t0);
        const uint32_t f = next_tile();
        TC_W_END(t0, 0);
        TC_W_BEGIN(b0);
        const uint32_t bs = bu % kAbuf;
        if (!f || *vabort || !mb_wait(afull + bs, (bu / kAbuf) & 1u, vabort, budget)) {
            fail();
            return;
        }
        TC_W_END(b0, 1);
        tc::fence_after_sync();
        TC_W_BEGIN(m0);
        mma_chunk(tm, tm + kAcol + 32 * bs, f, idesc, first);
        tc::mma_commit(cmb + gch % kCmb);
        TC_W_END(m0, 3);
        ++gch;
        ++bu;
    };
    // MMA thread: the accumulator is free (drained by the workers after its last use)
    auto wait_acc_free = [&]() {
        TC_W_BEGIN(a0);
        if (*vabort || !mb_wait(acce, (acnt & 1u) ^ 1u, vabort, budget)) fail();
        TC_W_END(a0, 2);
        tc::fence_after_sync();
    };
    // workers: write the operand block of chunk gch into tensor memory: the warp's 32 rows
    // (2 bl + comp), its 8 of the chunk's 16 complex columns, hi and lo parts.  v[u] is the
    // (already scaled) complex value of column 8 wh + u; conj selects the expansion:
    //   V^H X:  row 2b: (re, im), row 2b + 1: (im, -re)
    //   U Y:    row 2b: (re, -im), row 2b + 1: (im, re)
    auto build_block = [&](const float2 (&v)[8], bool vhx) {
        const uint32_t bs = bu % kAbuf;
        TC_W_BEGIN(w6);
        if (!*vabort && !chunk_done(buf_ch[bs])) fail();
        if (wt == 0) TC_W_END(w6, 6);
        buf_ch[bs] = gch;
        if (!warp_abort()) {
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float p0, p1;
                if (vhx) {
                    p0 = ocomp ? v[u].y : v[u].x;
                    p1 = ocomp ? -v[u].x : v[u].y;
                } else {
                    p0 = ocomp ? v[u].y : v[u].x;
                    p1 = ocomp ? v[u].x : -v[u].y;
                }
                // split both values at once (paired conversions): hi = fp16(p), lo = fp16(p - hi)
                const __half2 h = __floats2half2_rn(p0, p1);
                const float2 hb = __half22float2(h);
                const __half2 l = __floats2half2_rn(p0 - hb.x, p1 - hb.y);
                hi[u] = *reinterpret_cast<const uint32_t*>(&h);
                lo[u] = *reinterpret_cast<const uint32_t*>(&l);
            }
            const uint32_t ta = tm + ((uint32_t)(32 * wq) << 16) + kAcol + 32 * bs + 8 * wh;
            TC_W_BEGIN(w8);
            tc::tmem_st8(ta, hi);
            tc::tmem_st8(ta + 16, lo);
            if (wt == 0) TC_W_END(w8, 8);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(afull + bs);
        ++bu;
        ++gch;
    };

    // workers: the source values of chunk c (rows 16 c .. 16 c + 15 of X or of S o Y, the
    // warp's 8 of them, its 16 trajectories) into source slot k % kSrcSlots; each lane of
    // a pair copies 4 of the pair's 8 values, one completion group per chunk (empty past
    // the item's last chunk c_end).  Rows past N are zero-filled.
    float2* srcbuf = sDS;  // kSrcSlots x 8 KB, warp part (warp - 2) x 1 KB
    auto src_issue = [&](const float2* base, int c, int c_end, bool live, int b0, int k) {
        if (c < c_end) {
            float2* dst = srcbuf + (k % kSrcSlots) * 1024 + (warp - 2) * 128 + (obl & 15) * 8 + 4 * ocomp;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = (int64_t)c * 16 + 8 * wh + 4 * ocomp + u;
                const bool v = live && i < a.N;
                cp_async8(dst + u, v ? (const void*)(base + i * a.Bp + b0 + obl) : (const void*)base, v ? 8u : 0u);
            }
        }
        cp_async_commit();
    };
    // the same with the rows given by rowp(i): the row's base pointer, or null for a zero
    // row (channel-wise mode: gathered rows of X and of S o Y)
    auto src_issue_rows = [&](auto rowp, int c, int c_end, bool live, int b0, int k) {
        if (c < c_end) {
            float2* dst = srcbuf + (k % kSrcSlots) * 1024 + (warp - 2) * 128 + (obl & 15) * 8 + 4 * ocomp;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = (int64_t)c * 16 + 8 * wh + 4 * ocomp + u;
                const float2* row = live ? rowp(i) : nullptr;
                cp_async8(dst + u, row ? (const void*)(row + b0 + obl) : (const void*)a.X, row ? 8u : 0u);
            }
        }
        cp_async_commit();
    };
    // workers: wait for the source values of the chunk in slot k (kSrcAhead - 1 newer
    // groups may stay in flight) and read the pair's 8 values, scaled
    auto src_read = [&](float2 (&v)[8], int k, float sc) {
        TC_W_BEGIN(w7);
        cp_async_wait<kSrcAhead - 1>();
        __syncwarp();
        if (wt == 0) TC_W_END(w7, 7);
        const float2* src = srcbuf + (k % kSrcSlots) * 1024 + (warp - 2) * 128 + (obl & 15) * 8;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = make_float2(src[u].x * sc, src[u].y * sc);
        __syncwarp();  // the slot may be refilled after every lane has read it
    };

    for (int n = 0; n < a.Tmax && ok && (in_sync || producer); ++n) {
        const int Bact = a.act[a.n0 + n];
        const Groups q = stage_groups(a, Bact);
        for (int st = 0; st < 4 && ok; ++st) {
            const int gs = 4 * n + st;
            tr_gs = gs;
            const unsigned* xin = a.xmax + (gs % 3) * a.Bp;
            unsigned* xout = a.xmax + ((gs + 1) % 3) * a.Bp;
            TC_TRACE(worker && wt == 0, 0);
            if (blockIdx.x == 0 && worker)
                for (int b = wt; b < a.Bp; b += kWorkers) xout[b] = 0u;

            // ---------------- A: partials of V^H X ----------------
            const int nA = q.G * a.Mt * q.KS;
            if (producer) {
                for (int item = blockIdx.x; item < nA; item += gridDim.x) {
                    const ItemA it = item_a(a, q, item);
                    if constexpr (CHT) {
                        int qs, m;
                        seg_of_mt(a, it.m, qs, m);
                        const unsigned char* tv = a.tV + (a.tvoff[qs] + (int64_t)m * a.nchV) * kTile;
                        for (int c = it.c0; c < it.c1; ++c, ++gch) {
                            TC_W_BEGIN(p0);
                            issue(tv + (int64_t)c * kTile);
                            TC_W_END(p0, 4);
                        }
                    } else {
                        for (int c = it.c0; c < it.c1; ++c, ++gch) {
                            TC_W_BEGIN(p0);
                            issue(a.tV + ((int64_t)it.m * a.nchV + c) * kTile);
                            TC_W_END(p0, 4);
                        }
                    }
                }
            } else if (mma) {
                const uint32_t idesc = tc::idesc_f16(128, kRows);
                for (int item = blockIdx.x; item < nA && !*vabort; item += gridDim.x) {
                    const ItemA it = item_a(a, q, item);
                    wait_acc_free();
                    for (int c = it.c0; c < it.c1 && !*vabort; ++c) mma_step(idesc, c == it.c0);
                    tc::mma_commit(accf);
                    ++acnt;
                }
            } else if (worker) {
                for (int item = blockIdx.x; item < nA; item += gridDim.x) {
                    const ItemA it = item_a(a, q, item);
                    int b0, b1;
                    group_range(Bact, q.G, it.g, b0, b1);
                    const int nbg = b1 - b0;
                    workers_sync();  // the previous item's readers of ssc are done
                    if constexpr (CHT) {
                        if (wt < kGroup) ssc[wt] = wt < nbg ? pow2_scale(__uint_as_float(__ldcg(xin + b0 + wt))) : 0.f;
                    } else {
                        // the rows of this K-range: wait until every epilogue item of their row
                        // tiles has finished the previous stage, then this item's FP16 scale
                        // from the tiles' maxima
                        const int t0 = it.c0 * 16 / kRows, t1 = (it.c1 * 16 - 1) / kRows;
                        if (wt == 0 && a.use_flags && tdone_target > 0 && !*vabort) {
                            const uint64_t tw = gtimer();
                            for (int t = t0; t <= t1 && !*vabort; ++t)
                                while (ld_acquire64(a.tdone + t) < tdone_target) {
                                    if (gtimer() - tw > budget || *(volatile int*)a.err) {
                                        fail();
                                        break;
                                    }
                                    __nanosleep(32);
                                }
                        }
                        workers_sync();
                        if (wt < kGroup) {
                            unsigned mx = 0u;
                            if (wt < nbg)
                                for (int t = t0; t <= t1; ++t) mx = max(mx, __ldcg(a.xtile + (int64_t)t * a.Bp + b0 + wt));
                            ssc[wt] = wt < nbg ? pow2_scale(__uint_as_float(mx)) : 0.f;
                        }
                    }
                    workers_sync();
                    const float sx = ssc[obl];
                    const bool live = obl < nbg;
                    // X values of the warp's columns of chunk c, kSrcAhead chunks ahead
                    if constexpr (CHT) {
                        // rows k' P + q of X for the V segment q of this item
                        int qs, m;
                        seg_of_mt(a, it.m, qs, m);
                        const int P = a.npair, Nk = a.Nk;
                        auto rowx = [&](int64_t i) -> const float2* {
                            return i < Nk ? a.X + (i * P + qs) * a.Bp : nullptr;
                        };
                        for (int c = it.c0; c < it.c0 + kSrcAhead; ++c)
                            src_issue_rows(rowx, c, it.c1, live, b0, c - it.c0);
                        for (int c = it.c0; c < it.c1; ++c) {
                            float2 v[8];
                            src_read(v, c - it.c0, sx);
                            build_block(v, true);
                            src_issue_rows(rowx, c + kSrcAhead, it.c1, live, b0, c + kSrcAhead - it.c0);
                        }
                    } else {
                        for (int c = it.c0; c < it.c0 + kSrcAhead; ++c) src_issue(a.X, c, it.c1, live, b0, c - it.c0);
                        for (int c = it.c0; c < it.c1; ++c) {
                            float2 v[8];
                            src_read(v, c - it.c0, sx);
                            build_block(v, true);
                            src_issue(a.X, c + kSrcAhead, it.c1, live, b0, c + kSrcAhead - it.c0);
                        }
                    }
                    cp_async_wait<0>();
                    // accumulator -> raw partials P[ks][j][b]: lanes 2 bl and 2 bl + 1 hold the
                    // real and imaginary parts; the warp's half of the 256 columns (rows j)
                    if (!*vabort && !mb_wait(accf, acnt & 1u, vabort, budget)) fail();
                    tc::fence_after_sync();
                    if (!warp_abort()) {
                        float2* pbase = a.P + ((int64_t)it.ks * a.rp + (int64_t)it.m * kRows) * a.Bp + b0 + obl;
                        // low-rank mode: partials unscaled (each item has its own X scale)
                        const float ps = CHT ? 1.f : (live ? 1.f / (a.sv * sx) : 0.f);
                        for (int u = 0; u < 8; ++u) {
                            float v[16];
                            const int col = 128 * wh + 16 * u;
                            tc::tmem_ld16(tm + ((uint32_t)(32 * wq) << 16) + col, v);
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                const float im = __shfl_xor_sync(0xffffffffu, v[t], 1);
                                if (!ocomp && live) pbase[(int64_t)(col + t) * a.Bp] = make_float2(v[t] * ps, im * ps);
                            }
                        }
                    }
                    tc::fence_before_sync();
                    mbar_arrive(acce);
                    ++acnt;
                }
            }
            TC_TRACE(worker && wt == 0, 1);
            if (in_sync && !(ok = tc_grid_sync(a, gen, &abort_s))) break;
            TC_TRACE(worker && wt == 0, 2);
            if (st == 0 && a.ckS && worker && (a.n0 + n) % a.ck_period == 0) {
                // checkpoint of the compensated state at the start of step n0 + n (every
                // epilogue of the previous step is complete after the first barrier; stable
                // until the last stage's epilogue of this step)
                const int64_t slot = (int64_t)((a.n0 + n) / a.ck_period) * a.N * a.Bp;
                const int64_t tot = a.N * Bact;
                for (int64_t e = (int64_t)blockIdx.x * kWorkers + wt; e < tot; e += (int64_t)gridDim.x * kWorkers) {
                    const int64_t off = (e / Bact) * a.Bp + e % Bact;
                    a.ckS[slot + off] = __ldcg(a.Ssum + off);
                    a.ckC[slot + off] = __ldcg(a.Ccomp + off);
                }
            }

            // ---------------- B: S o sum of the partials, scaled for FP16 ----------------
            if (worker) {
                const int64_t gt = (int64_t)blockIdx.x * kWorkers + wt, total = (int64_t)gridDim.x * kWorkers;
                if constexpr (CHT) {
                    const int64_t tot_el = (int64_t)a.rp * Bact;
                    for (int64_t e = gt; e < tot_el; e += total) {
                        const int j = (int)(e / Bact), b = (int)(e % Bact);
                        float2 v = make_float2(0.f, 0.f);
                        // column of S: the padded column j is column jj of V segment qs
                        int qs, m;
                        seg_of_mt(a, j / kRows, qs, m);
                        const int jj = m * kRows + j % kRows;
                        const int sj = jj < a.ldvq[qs] ? a.sbq[qs] + jj : -1;
                        if (sj >= 0) {
                            // eight independent partial sums (loads in flight), fixed order
                            const float2* pp = a.P + (int64_t)j * a.Bp + b;
                            const int64_t pstride = (int64_t)a.rp * a.Bp;
                            float2 s8[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) s8[u] = make_float2(0.f, 0.f);
                            int k2 = 0;
                            for (; k2 + 8 <= q.KS; k2 += 8) {
#pragma unroll
                                for (int u = 0; u < 8; ++u) s8[u] = cadd(s8[u], __ldcg(pp + (k2 + u) * pstride));
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (k2 + u < q.KS) s8[u] = cadd(s8[u], __ldcg(pp + (k2 + u) * pstride));
                            const float2 s = cadd(cadd(cadd(s8[0], s8[1]), cadd(s8[2], s8[3])),
                                                  cadd(cadd(s8[4], s8[5]), cadd(s8[6], s8[7])));
                            // unscaled: the U-pass operand mixes S o y and x, scaled together
                            const float mx = __uint_as_float(__ldcg(xin + b));
                            v = cscale(s, a.S[sj] * (1.f / (a.sv * pow2_scale(mx))));
                        }
                        a.Ys[(int64_t)j * a.Bp + b] = v;
                    }
                } else {
                    const int64_t tot_el = (int64_t)a.rp * Bact;
                    for (int64_t e = gt; e < tot_el; e += total) {
                        const int j = (int)(e / Bact), b = (int)(e % Bact);
                        float2 v = make_float2(0.f, 0.f);
                        if (j < a.r) {
                            // eight independent partial sums (loads in flight), fixed order
                            const float2* pp = a.P + (int64_t)j * a.Bp + b;
                            const int64_t pstride = (int64_t)a.rp * a.Bp;
                            float2 s8[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) s8[u] = make_float2(0.f, 0.f);
                            int k2 = 0;
                            for (; k2 + 8 <= q.KS; k2 += 8) {
#pragma unroll
                                for (int u = 0; u < 8; ++u) s8[u] = cadd(s8[u], __ldcg(pp + (k2 + u) * pstride));
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (k2 + u < q.KS) s8[u] = cadd(s8[u], __ldcg(pp + (k2 + u) * pstride));
                            const float2 s = cadd(cadd(cadd(s8[0], s8[1]), cadd(s8[2], s8[3])),
                                                  cadd(cadd(s8[4], s8[5]), cadd(s8[6], s8[7])));
                            const float mx = __uint_as_float(__ldcg(xin + b));
                            v = cscale(s, a.S[j] * pow2_scale(a.ybound * mx));
                        }
                        a.Ys[(int64_t)j * a.Bp + b] = v;
                    }
                }
                if (CHT && st == 0 && n > 0) {
                    tc_obs_warp(a, n, blockIdx.x * (kWorkers / 32) + (warp - 2), gridDim.x * (kWorkers / 32), lane);
                } else if (st == 0 && n > 0) {
                    // observables of step n (written by the last stage of step n - 1)
                    for (int64_t b = gt; b < a.act[a.n0 + n - 1]; b += total) {
                        double s0 = 0, s1 = 0, s2 = 0;
                        for (int t = 0; t < a.Nred; ++t) {
                            const double* rr = a.red + ((int64_t)t * a.Bp + b) * 3;
                            s0 += __ldcg(rr);
                            s1 += __ldcg(rr + 1);
                            s2 += __ldcg(rr + 2);
                        }
                        double* o = a.obs + ((int64_t)n * a.B + b) * 3;
                        o[0] = s0 / a.Nk;
                        o[1] = s1 / a.Nk;
                        o[2] = s2 / a.Nk;
                    }
                }
            }
            TC_TRACE(worker && wt == 0, 3);
            if (in_sync && !(ok = tc_grid_sync(a, gen, &abort_s))) break;
            TC_TRACE(worker && wt == 0, 4);

            // ---------------- C: dSigma = U (S o Y) + K^diag o X, commutator, RK4 ----------------
            const int eoff = st == 0 ? 0 : (st == 3 ? 2 : 1);
            if constexpr (!CHT) {
                const int nC = a.Nt * q.GC;
                if (producer) {
                    for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                        const int t = item % a.Nt;
                        for (int c = 0; c < a.nchU; ++c, ++gch) {
                            TC_W_BEGIN(p1);
                            issue(a.tU + ((int64_t)t * a.nchU + c) * kTile);
                            TC_W_END(p1, 4);
                        }
                    }
                    TC_TRACE(true, 8);
                } else if (mma) {
                    const uint32_t idesc = tc::idesc_f16(128, kRows);
                    for (int item = blockIdx.x; item < nC && !*vabort; item += gridDim.x) {
                        wait_acc_free();
                        for (int c = 0; c < a.nchU && !*vabort; ++c) mma_step(idesc, c == 0);
                        tc::mma_commit(accf);
                        ++acnt;
                    }
                    TC_TRACE(true, 7);
                } else if (worker) {
                    for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                        const int t = item % a.Nt, g = item / a.Nt;
                        int b0, b1;
                        group_range(Bact, q.GC, g, b0, b1);
                        const int nbg = b1 - b0;
                        workers_sync();  // the previous item's readers of ssc, smx, sred are done
                        if (wt < kGroup) {
                            if (wt < nbg) {
                                const float mx = __uint_as_float(__ldcg(xin + b0 + wt));
                                ssc[wt] = 1.f / (a.su * pow2_scale(a.ybound * mx));
                            }
                            smx[wt] = 0u;
                        }
                        workers_sync();
                        const bool live = obl < nbg;
                        // S o Y values of the warp's columns of chunk c, kSrcAhead chunks ahead
                        for (int c = 0; c < kSrcAhead; ++c) src_issue(a.Ys, c, a.nchU, live, b0, c);
                        for (int c = 0; c < a.nchU; ++c) {
                            float2 v[8];
                            src_read(v, c, 1.f);
                            build_block(v, false);
                            src_issue(a.Ys, c + kSrcAhead, a.nchU, live, b0, c + kSrcAhead);
                        }
                        cp_async_wait<0>();
                        if (!*vabort && !mb_wait(accf, acnt & 1u, vabort, budget)) fail();
                        tc::fence_after_sync();
                        const int kgroups = kWorkers / nbg;
                        const int bl = wt % nbg, kg = wt / nbg;
                        DF3 obs;
                        float xm = 0.f;
                        for (int qq = 0; qq < kRows / 64; ++qq) {
                            // accumulator columns 64 qq .. + 63 (the warp's 32 of them) -> staged
                            // quarter, unscaled; lanes 2 bl and 2 bl + 1 hold re and im
                            if (!warp_abort()) {
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    float v[16];
                                    const int col = 64 * qq + 32 * wh + 16 * u;
                                    tc::tmem_ld16(tm + ((uint32_t)(32 * wq) << 16) + col, v);
                                    const float sc = live ? ssc[obl] : 0.f;
#pragma unroll
                                    for (int e = 0; e < 16; ++e) {
                                        const float im = __shfl_xor_sync(0xffffffffu, v[e], 1);
                                        if (!ocomp && live)
                                            sDS[ds_index(32 * wh + 16 * u + e, obl)] = make_float2(v[e] * sc, im * sc);
                                    }
                                }
                            }
                            workers_sync();
                            // commutator + RK4 for the k-blocks of these 64 rows
                            const int kbase = (t * kRows + 64 * qq) / NB2;
                            const int kt = min(64 / NB2, a.Nk - kbase);
                            if (kg < kgroups && !*vabort) {
                                const int b = b0 + bl;
                                const float E = (float)a.Etab[(int64_t)b * a.ldE + 2 * (a.n0 + n) + eoff];
                                const float2 dr = a.dir[b];
                                const int64_t rec = a.recX ? (int64_t)(4 * n + st) * a.N * a.Bp : -1;
                                for (int kl = kg; kl < kt; kl += kgroups)
                                    stage_kb_tc<NB>(a, kbase + kl, b, st, E, dr, sDS, kl * NB2, bl, xm, obs, rec);
                            }
                            workers_sync();  // the staged quarter is consumed before it is rewritten
                        }
                        tc::fence_before_sync();
                        mbar_arrive(acce);
                        ++acnt;
                        if (kg < kgroups) {
                            atomicMax(smx + bl, __float_as_uint(xm));
                            if (st == 3) {
                                sred[(kg * nbg + bl) * 3] = obs.p.value();
                                sred[(kg * nbg + bl) * 3 + 1] = obs.j.value();
                                sred[(kg * nbg + bl) * 3 + 2] = obs.o.value();
                            }
                        }
                        workers_sync();
                        if (wt < nbg && !*vabort) {
                            atomicMax(xout + b0 + wt, smx[wt]);
                            a.xtile[(int64_t)t * a.Bp + b0 + wt] = smx[wt];
                            if (st == 3) {
                                double r0 = 0.0, r1 = 0.0, r2 = 0.0;
                                for (int k2 = 0; k2 < kgroups; ++k2) {
                                    r0 += sred[(k2 * nbg + wt) * 3];
                                    r1 += sred[(k2 * nbg + wt) * 3 + 1];
                                    r2 += sred[(k2 * nbg + wt) * 3 + 2];
                                }
                                double* rr = a.red + ((int64_t)t * a.Bp + b0 + wt) * 3;
                                rr[0] = r0;
                                rr[1] = r1;
                                rr[2] = r2;
                            }
                        }
                        // every row of this item is written: count it for the tile (release)
                        workers_sync();
                        if (wt == 0) red_release_add64(a.tdone + t, 1ull);
                    }
                }
            } else {
                // ---- C (channel-wise): dSigma rows k P + p of U segment p's row tile t ----
                // items: (segment tile si = p NtK + t, trajectory group g, K-range kc)
                const int nC = a.Nt * q.GC * a.kcu;  // a.Nt: P NtK segment tiles
                auto item_c = [&](int item, int& p, int& t, int& g, int& kc, int& c0, int& c1) {
                    const int si = item % a.Nt, rest = item / a.Nt;
                    p = si / a.NtK;
                    t = si % a.NtK;
                    g = rest % q.GC;
                    kc = rest / q.GC;
                    c0 = a.nchw[p] * kc / a.kcu;
                    c1 = a.nchw[p] * (kc + 1) / a.kcu;
                };
                if (producer) {
                    for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                        int p, t, g, kc, c0, c1;
                        item_c(item, p, t, g, kc, c0, c1);
                        const unsigned char* tu = a.tU + (a.tuoff[p] + (int64_t)t * a.nchw[p]) * kTile;
                        for (int c = c0; c < c1; ++c, ++gch) {
                            TC_W_BEGIN(p1);
                            issue(tu + (int64_t)c * kTile);
                            TC_W_END(p1, 4);
                        }
                    }
                    TC_TRACE(true, 8);
                } else if (mma) {
                    const uint32_t idesc = tc::idesc_f16(128, kRows);
                    for (int item = blockIdx.x; item < nC && !*vabort; item += gridDim.x) {
                        int p, t, g, kc, c0, c1;
                        item_c(item, p, t, g, kc, c0, c1);
                        wait_acc_free();
                        for (int c = c0; c < c1 && !*vabort; ++c) mma_step(idesc, c == c0);
                        tc::mma_commit(accf);
                        ++acnt;
                    }
                } else if (worker) {
                    for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                        int p, t, g, kc, c0, c1;
                        item_c(item, p, t, g, kc, c0, c1);
                        int b0, b1;
                        group_range(Bact, q.GC, g, b0, b1);
                        const int nbg = b1 - b0;
                        workers_sync();  // the previous item's readers of ssc are done
                        if (wt < kGroup && wt < nbg) ssc[wt] = pow2_scale(a.zbound * __uint_as_float(__ldcg(xin + b0 + wt)));
                        workers_sync();
                        const bool live = obl < nbg;
                        const float sz = live ? ssc[obl] : 0.f;
                        // operand z_p: the S o y rows of the channels out of p, then x_p
                        const int nl = a.nlrq[p], P = a.npair, Nk = a.Nk;
                        const int* gp = a.gpad + a.gbq[p];
                        auto rowz = [&](int64_t j) -> const float2* {
                            if (j < nl) return a.Ys + (int64_t)__ldg(gp + j) * a.Bp;
                            return j < nl + Nk ? a.X + ((j - nl) * P + p) * a.Bp : nullptr;
                        };
                        for (int c = c0; c < c0 + kSrcAhead; ++c) src_issue_rows(rowz, c, c1, live, b0, c - c0);
                        for (int c = c0; c < c1; ++c) {
                            float2 v[8];
                            src_read(v, c - c0, sz);
                            build_block(v, false);
                            src_issue_rows(rowz, c + kSrcAhead, c1, live, b0, c + kSrcAhead - c0);
                        }
                        cp_async_wait<0>();
                        // accumulator -> partial dSigma rows k P + p of K-range kc (unscaled);
                        // lanes 2 bl and 2 bl + 1 hold the real and imaginary parts
                        if (!*vabort && !mb_wait(accf, acnt & 1u, vabort, budget)) fail();
                        tc::fence_after_sync();
                        if (!warp_abort()) {
                            // an empty K-range (fewer chunks than ranges) contributes zeros
                            const float osc = live && c1 > c0 ? 1.f / (a.su * sz) : 0.f;
                            for (int u = 0; u < 8; ++u) {
                                float v[16];
                                const int col = 128 * wh + 16 * u;
                                tc::tmem_ld16(tm + ((uint32_t)(32 * wq) << 16) + col, v);
#pragma unroll
                                for (int e = 0; e < 16; ++e) {
                                    const float im = __shfl_xor_sync(0xffffffffu, v[e], 1);
                                    const int k = t * kRows + col + e;
                                    if (!ocomp && live && k < Nk)
                                        a.dS[((int64_t)kc * a.N + (int64_t)k * P + p) * a.Bp + b0 + obl] =
                                            make_float2(v[e] * osc, im * osc);
                                }
                            }
                        }
                        tc::fence_before_sync();
                        mbar_arrive(acce);
                        ++acnt;
                    }
                }
                // every dSigma row is written before the epilogue reads it
                if (in_sync && !(ok = tc_grid_sync(a, gen, &abort_s))) break;
                TC_TRACE(worker && wt == 0, 7);
                // ---- E (channel-wise): commutator + RK4 by 64-row quarters of all N rows
                //      (items: quarter, trajectory group), dSigma summed over the K-range
                //      partials of phase C in a fixed order into the staging buffer ----
                if (worker) {
                    const int nq = 4 * a.nte;
                    const int nE = nq * q.GC;
                    for (int item = blockIdx.x; item < nE; item += gridDim.x) {
                        const int tq = item % nq, g = item / nq;
                        int b0, b1;
                        group_range(Bact, q.GC, g, b0, b1);
                        const int nbg = b1 - b0;
                        workers_sync();  // the previous item's readers of smx and sred are done
                        if (wt < kGroup) smx[wt] = 0u;
                        const int64_t r0 = (int64_t)tq * 64;
                        for (int e = wt; e < 64 * nbg; e += kWorkers) {
                            const int rr = e / nbg, bb = e % nbg;
                            if (r0 + rr < a.N) {
                                const float2* src = a.dS + (r0 + rr) * a.Bp + b0 + bb;
                                float2 v = __ldcg(src);
                                for (int kc = 1; kc < a.kcu; ++kc) v = cadd(v, __ldcg(src + (int64_t)kc * a.N * a.Bp));
                                sDS[ds_index(rr, bb)] = v;
                            }
                        }
                        workers_sync();
                        const int kgroups = kWorkers / nbg;
                        const int bl = wt % nbg, kg = wt / nbg;
                        DF3 obs;
                        float xm = 0.f;
                        const int kbase = (int)(r0 / NB2);
                        const int kt = min(64 / NB2, a.Nk - kbase);
                        if (kg < kgroups && !*vabort) {
                            const int b = b0 + bl;
                            const float E = (float)a.Etab[(int64_t)b * a.ldE + 2 * (a.n0 + n) + eoff];
                            const float2 dr = a.dir[b];
                            for (int kl = kg; kl < kt; kl += kgroups)
                                stage_kb_tc<NB>(a, kbase + kl, b, st, E, dr, sDS, kl * NB2, bl, xm, obs, -1);
                        }
                        workers_sync();  // the staged quarter is consumed before sred reuses it
                        if (kg < kgroups) {
                            atomicMax(smx + bl, __float_as_uint(xm));
                            if (st == 3) {
                                sred[(kg * nbg + bl) * 3] = obs.p.value();
                                sred[(kg * nbg + bl) * 3 + 1] = obs.j.value();
                                sred[(kg * nbg + bl) * 3 + 2] = obs.o.value();
                            }
                        }
                        workers_sync();
                        if (wt < nbg && !*vabort) {
                            atomicMax(xout + b0 + wt, smx[wt]);
                            if (st == 3) {
                                double r0s = 0.0, r1s = 0.0, r2s = 0.0;
                                for (int k2 = 0; k2 < kgroups; ++k2) {
                                    r0s += sred[(k2 * nbg + wt) * 3];
                                    r1s += sred[(k2 * nbg + wt) * 3 + 1];
                                    r2s += sred[(k2 * nbg + wt) * 3 + 2];
                                }
                                double* rr = a.red + ((int64_t)tq * a.Bp + b0 + wt) * 3;
                                rr[0] = r0s;
                                rr[1] = r1s;
                                rr[2] = r2s;
                            }
                        }
                    }
                }
            }
            TC_TRACE(worker && wt == 0, 5);
            if (CHT || !a.use_flags) {
                if (in_sync) ok = tc_grid_sync(a, gen, &abort_s);
            } else {
                // no grid barrier: the next stage's phase A items wait for their row tiles (an
                // abort is seen uniformly at the next stage's first barrier)
                tdone_target += (unsigned long long)q.GC;
            }
            TC_TRACE(worker && wt == 0, 6);
        }
    }
    // observables of the last step (workers: they passed the last grid barrier)
    // low-rank mode: every CTA's last epilogue is complete before the last observables
    if (!CHT && in_sync && ok && a.Tmax > 0) ok = tc_grid_sync(a, gen, &abort_s);
    if (CHT && worker && ok && a.Tmax > 0) {
        tc_obs_warp(a, a.Tmax, blockIdx.x * (kWorkers / 32) + (warp - 2), gridDim.x * (kWorkers / 32), lane);
    } else if (worker && ok && a.Tmax > 0) {
        const int n = a.Tmax;
        const int64_t gt = (int64_t)blockIdx.x * kWorkers + wt, total = (int64_t)gridDim.x * kWorkers;
        for (int64_t b = gt; b < a.act[a.n0 + n - 1]; b += total) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int t = 0; t < a.Nred; ++t) {
                const double* rr = a.red + ((int64_t)t * a.Bp + b) * 3;
                s0 += __ldcg(rr);
                s1 += __ldcg(rr + 1);
                s2 += __ldcg(rr + 2);
            }
            double* o = a.obs + ((int64_t)n * a.B + b) * 3;
            o[0] = s0 / a.Nk;
            o[1] = s1 / a.Nk;
            o[2] = s2 / a.Nk;
        }
    }
    // teardown: no copy and no MMA of this CTA may remain in flight (after an abort some
    // issued tiles may never have been consumed)
    if (producer) {
        const uint32_t first = ppos > (uint32_t)kRing ? ppos - kRing : 0u;
        for (uint32_t p = first; p < ppos; ++p) mb_wait(full + p % kRing, (p / kRing) & 1u, nullptr, budget);
    }
    if (mma) {
        tc::mma_commit(fin);
        mb_wait(fin, 0u, nullptr, budget);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, kTmemCols);
    }
}

// max(|Re|, |Im|) of each trajectory's stage input X over each 256-row tile, as float bits
// (block (t, b)): the per-tile maxima of a launch that starts from a restored state
__global__ void xtile_kernel(const float2* __restrict__ X, int64_t N, int Bp, unsigned* __restrict__ xtile) {
    const int t = blockIdx.x, b = blockIdx.y;
    float m = 0.f;
    for (int r = threadIdx.x; r < kRows; r += blockDim.x) {
        const int64_t i = (int64_t)t * kRows + r;
        if (i < N) {
            const float2 v = X[i * Bp + b];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
        m = fmaxf(m, wm[0]);
        xtile[(int64_t)t * Bp + b] = __float_as_uint(m);
    }
}

// max(|Re|, |Im|) of each trajectory's stage input X (N x Bp) as float bits, into xmax
// (zeroed by the caller): the split-FP16 scale of a launch that starts from a restored state.
__global__ void xmax_kernel(const float2* __restrict__ X, int64_t N, int Bp, unsigned* __restrict__ xmax) {
    const int b = blockIdx.y;
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = X[i * Bp + b];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(xmax + b, __float_as_uint(m));
}

// Per column j: max(|Re|, |Im|) of U and of V, and ||v_j||^2.
__global__ void factor_stats_kernel(const float2* __restrict__ U, const float2* __restrict__ V, int64_t N,
                                    int r, int ldu, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= r) return;
    float mu = 0.f, mv = 0.f;
    double nv = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const float2 u = U[i * ldu + j], v = V[i * ldu + j];
        mu = fmaxf(mu, fmaxf(fabsf(u.x), fabsf(u.y)));
        mv = fmaxf(mv, fmaxf(fabsf(v.x), fabsf(v.y)));
        nv += (double)v.x * v.x + (double)v.y * v.y;
    }
    out[j] = mu;
    out[r + j] = mv;
    out[2 * r + j] = (float)nv;
}

// Split-FP16 tiles of U: tile (t, c) holds rows 256 t .. +255 and complex columns
// 16 c .. +15 as 32 real columns (re, im), scaled by `scale`; zero outside N x r.
__global__ void pack_u_kernel(const float2* __restrict__ U, int64_t N, int r, int ldu, int rp, int nchU,
                              float scale, unsigned char* __restrict__ out, int64_t total) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t i = e / rp;
    const int j = (int)(e % rp);
    float2 v = make_float2(0.f, 0.f);
    if (i < N && j < r) v = U[i * ldu + j];
    __half rh, rl, ih, il;
    split16(v.x * scale, rh, rl);
    split16(v.y * scale, ih, il);
    unsigned char* tile = out + ((i / kRows) * nchU + j / 16) * (int64_t)kTile;
    const uint32_t o = tc::kmajor_offset((uint32_t)(i % kRows), 2 * (j % 16), kKc);
    *reinterpret_cast<__half2*>(tile + o) = __halves2half2(rh, ih);
    *reinterpret_cast<__half2*>(tile + kHalf + o) = __halves2half2(rl, il);
}

// Split-FP16 tiles of V^T: tile (m, c) holds rows j = 256 m .. +255 (columns of V) and
// rows i = 16 c .. +15 of V as 32 real columns (re, im), scaled by `scale`.
__global__ void pack_v_kernel(const float2* __restrict__ V, int64_t N, int r, int ldu, int rp, int nchV,
                              float scale, unsigned char* __restrict__ out, int64_t total) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t i = e / rp;
    const int j = (int)(e % rp);
    float2 v = make_float2(0.f, 0.f);
    if (i < N && j < r) v = V[i * ldu + j];
    __half rh, rl, ih, il;
    split16(v.x * scale, rh, rl);
    split16(v.y * scale, ih, il);
    unsigned char* tile = out + ((int64_t)(j / kRows) * nchV + i / 16) * (int64_t)kTile;
    const uint32_t o = tc::kmajor_offset((uint32_t)(j % kRows), (uint32_t)(2 * (i % 16)), kKc);
    *reinterpret_cast<__half2*>(tile + o) = __halves2half2(rh, ih);
    *reinterpret_cast<__half2*>(tile + kHalf + o) = __halves2half2(rl, il);
}

struct TcDims {
    int Nt, Np, rp, Mt, nchU, nchV;
};
TcDims tc_dims(int64_t N, int r) {
    TcDims d;
    d.Nt = (int)((N + kRows - 1) / kRows);
    d.Np = d.Nt * kRows;
    d.rp = (r + kRows - 1) / kRows * kRows;
    d.Mt = d.rp / kRows;
    d.nchU = 2 * d.rp / kKc;
    d.nchV = 2 * d.Np / kKc;
    return d;
}

size_t tc_smem_bytes() {
    static_assert(kWorkers * 3 * sizeof(double) <= kStg, "observable sums fit the staging buffer");
    return (size_t)kRing * kTile + kStg + kGroup * sizeof(float) + kGroup * sizeof(unsigned) +
           (kRing + kCmb + kAbuf + 3) * sizeof(uint64_t);
}

}  // namespace

#ifdef TDAGW_TRACE
extern "C" int tdagw_debug_trace_tc(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_trace_tc, sizeof(unsigned long long) * (size_t)n) == cudaSuccess ? 0 : -3;
}
extern "C" int tdagw_debug_trace_tc_w(unsigned long long* out) {
    return cudaMemcpyFromSymbol(out, g_trace_w, sizeof(unsigned long long) * 160 * kTraceStages * 9) == cudaSuccess ? 0 : -3;
}
#endif

void pack_factors_tc(Ctx& c) {
    if (c.tc_valid) return;
    TDAGW_REQUIRE(c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED, "split-FP16 factors need a complex64 context");
    TDAGW_REQUIRE(c.rank > 0, TDAGW_ERR_NO_FACTORS, "no low-rank factors installed");
    cudaStream_t s = c.stream;
    const int64_t N = c.hm.N;
    const int r = c.rank, ldu = r + (r & 1);
    const TcDims d = tc_dims(N, r);
    const int64_t total = (int64_t)d.Np * d.rp;
    c.tcU.ensure((size_t)d.Nt * d.nchU * kTile);
    c.tcV.ensure((size_t)d.Mt * d.nchV * kTile);
    // magnitudes of the factors: power-of-two tile scales and the bound of S o Y
    DevBuf stats;
    stats.ensure((size_t)3 * r * sizeof(float));
    factor_stats_kernel<<<(r + 127) / 128, 128, 0, s>>>(c.U.as<float2>(), c.V.as<float2>(), N, r, ldu,
                                                       stats.as<float>());
    check_launch("factor_stats_kernel");
    std::vector<float> st(3 * (size_t)r), S(r);
    TDAGW_CUDA(cudaMemcpyAsync(st.data(), stats.p, st.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    TDAGW_CUDA(cudaMemcpyAsync(S.data(), c.S.p, r * sizeof(float), cudaMemcpyDeviceToHost, s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
    float mu = 0.f, mv = 0.f, nv = 0.f, smax = 0.f;
    for (int j = 0; j < r; ++j) {
        mu = std::max(mu, st[j]);
        mv = std::max(mv, st[r + j]);
        nv = std::max(nv, st[2 * r + j]);
        smax = std::max(smax, std::fabs(S[j]));
    }
    TDAGW_REQUIRE(std::isfinite(mu) && std::isfinite(mv) && std::isfinite(nv) && std::isfinite(smax),
                  TDAGW_ERR_INVALID_ARG, "factors are not finite");
    auto p2 = [](float bound) {
        if (!(bound > 0.f)) return 1.f;
        int e = 0;
        std::frexp(bound, &e);
        return std::ldexp(1.f, 13 - std::max(e, -100));
    };
    c.tc_su = p2(mu);
    c.tc_sv = p2(mv);
    c.tc_ybound = smax * std::sqrt(nv) * (float)std::sqrt(2.0 * (double)N);
    const unsigned blocks = (unsigned)((total + 255) / 256);
    pack_u_kernel<<<blocks, 256, 0, s>>>(c.U.as<float2>(), N, r, ldu, d.rp, d.nchU, c.tc_su,
                                         c.tcU.as<unsigned char>(), total);
    check_launch("pack_u_kernel");
    pack_v_kernel<<<blocks, 256, 0, s>>>(c.V.as<float2>(), N, r, ldu, d.rp, d.nchV, c.tc_sv,
                                         c.tcV.as<unsigned char>(), total);
    check_launch("pack_v_kernel");
    TDAGW_CUDA(cudaStreamSynchronize(s));
    c.tc_valid = true;
}

void propagate_batched_tc(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt, int flags) {
    TDAGW_REQUIRE(c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED, "split-FP16 propagation needs a complex64 context");
    TDAGW_REQUIRE(flags & TDAGW_FLAG_RESET, TDAGW_ERR_UNSUPPORTED,
                  "split-FP16 propagation starts from drho = 0 (TDAGW_FLAG_RESET)");
    pack_factors_tc(c);
    const HostModel& h = c.hm;
    cudaStream_t s = c.stream;
    const int64_t N = h.N;
    const int r = c.rank;
    const TcDims d = tc_dims(N, r);
    const BatchSetup bs = prepare_batch(c, fields, B, steps, dt);
    const int Bp = bs.Bp;

    int dev = 0, nsm = 0;
    TDAGW_CUDA(cudaGetDevice(&dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = tc_smem_bytes();
    const void* fn = h.Nb == 2 ? (const void*)batched_tc_kernel<2, false> : (const void*)batched_tc_kernel<4, false>;
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, smem));
    TDAGW_REQUIRE(per_sm == 1, TDAGW_ERR_UNSUPPORTED, "tensor-core batched kernel needs exactly one CTA per SM");
    const int nctas = nsm;

    // largest split of the V^H X reduction over the run (one trajectory group)
    const int KSmax = std::max(1, std::min(nctas / d.Mt, d.nchV));
    c.tcP.ensure((size_t)KSmax * d.rp * Bp * sizeof(float2));
    c.tcY.ensure((size_t)d.rp * Bp * sizeof(float2));
    c.tcMax.ensure((size_t)3 * Bp * sizeof(unsigned));
    c.tcRed.ensure((size_t)d.Nt * Bp * 3 * sizeof(double));
    c.tcDone.ensure((size_t)d.Nt * sizeof(unsigned long long));
    c.tcXt.ensure((size_t)d.Nt * Bp * sizeof(unsigned));
    const size_t sbytes = (size_t)N * Bp * sizeof(float2);
    c.sync.ensure(4 * sizeof(unsigned));

    TcArgs a{};
    a.tU = c.tcU.as<unsigned char>();
    a.tV = c.tcV.as<unsigned char>();
    a.Ys = c.tcY.as<float2>();
    a.P = c.tcP.as<float2>();
    a.xmax = c.tcMax.as<unsigned>();
    a.S = c.S.as<float>();
    a.diag = c.diagF.as<float2>();
    a.dx = c.dx.as<float2>();
    a.dy = c.dy.as<float2>();
    a.vx = c.vx.as<float2>();
    a.gap = c.gap.as<float2>();
    a.X = c.bX.as<float2>();
    a.Ssum = c.bS.as<float2>();
    a.Ccomp = c.bC.as<float2>();
    a.acc = c.bA.as<float2>();
    a.Etab = c.bEtab.as<double>();
    a.dir = c.bdir.as<float2>();
    a.act = c.bact.as<int>();
    a.red = c.tcRed.as<double>();
    a.obs = c.bobs.as<double>();
    a.bar = reinterpret_cast<unsigned long long*>(c.sync.p);
    a.err = reinterpret_cast<int*>(c.sync.as<unsigned>() + 2);
    a.tdone = c.tcDone.as<unsigned long long>();
    a.xtile = c.tcXt.as<unsigned>();
    a.N = N;
    a.ldE = bs.ldE;
    a.Nk = h.Nk;
    a.r = r;
    a.rp = d.rp;
    a.Nt = d.Nt;
    a.Nred = d.Nt;
    a.Mt = d.Mt;
    a.nchU = d.nchU;
    a.nchV = d.nchV;
    a.Bp = Bp;
    a.B = B;
    a.kahan = (flags & TDAGW_FLAG_NO_KAHAN) ? 0 : 1;
    a.c1 = h.c1;
    for (int q = 0; q < 4; ++q) a.occ[q] = (float)h.occ[q];
    a.dt = (float)dt;
    a.su = c.tc_su;
    a.sv = c.tc_sv;
    a.ybound = c.tc_ybound;
    a.wait_ns = 2000000000ull;
    a.n0 = 0;
    a.ck_period = 1;
    const bool ckpt = (flags & TDAGW_FLAG_CHECKPOINT) != 0;
    int period = 1;
    if (ckpt) {
        // compensated state every ceil(sqrt(Tmax)) steps for the adjoint's recomputes
        period = std::max(1, (int)std::ceil(std::sqrt((double)bs.Tmax)));
        const int nck = (bs.Tmax + period - 1) / period;
        c.ckS.ensure((size_t)nck * sbytes);
        c.ckC.ensure((size_t)nck * sbytes);
    }
    auto run = [&](int gc_max, int ks_max, int fl, int T, bool graph) {
        a.gc_max = gc_max;
        a.ks_max = ks_max;
        a.use_flags = fl;
        a.Tmax = T;
        launch_batched(c, fn, dim3(nctas), dim3(kTcThreads), smem, &a, sizeof(a),
                       {{c.bX.p, sbytes},
                        {c.bS.p, sbytes},
                        {c.bC.p, sbytes},
                        {c.tcMax.p, 3 * Bp * sizeof(unsigned)},
                        {c.tcDone.p, d.Nt * sizeof(unsigned long long)},
                        {c.tcXt.p, d.Nt * Bp * sizeof(unsigned)},
                        {c.sync.p, 4 * sizeof(unsigned)}},
                       graph);
    };

    // Work split of the launch, tuned once per (B, rank) on this context by timing a few
    // steps of each candidate: the trajectory groups of the U product (fewer groups stream
    // U fewer times and waste fewer MMA rows; more groups fill more CTAs when N is small),
    // the K-ranges of the V^H X product (all CTAs, or half as many longer ranges with half
    // the partial sums), and whether the next stage's V^H X items wait for their row tiles
    // through per-tile counters or all CTAs meet at a grid barrier after the epilogue.
    const uint64_t key = (0xF0ull << 56) | ((uint64_t)B << 32) | (uint64_t)(uint32_t)r;
    int gc_max = 0, ks_max = 0, flags_on = 1;
    const bool test_timeout = (flags & TDAGW_FLAG_TEST_TIMEOUT) != 0;
    auto it = c.batch_plans.find(key);
    if (test_timeout) {
        // timeout test: no tuning; the launch below waits for an arrival that never comes
    } else if (it != c.batch_plans.end()) {
        gc_max = it->second.first;
        ks_max = it->second.second & 0xFFFFF;
        flags_on = it->second.second >> 20;
    } else {
        const int g_min = (B + kGroup - 1) / kGroup;
        const int g_fill = group_count(B, d.Nt, nctas, 0);
        std::vector<int> gcs;
        for (int gcand = g_min; gcand < g_fill; gcand *= 2) gcs.push_back(gcand);
        gcs.push_back(0);
        const int ks_fill = std::max(1, std::min(nctas / (g_min * d.Mt), d.nchV));
        std::vector<int> kss = {0};
        if (ks_fill >= 4) kss.push_back(ks_fill / 2);
        if (bs.Tmax >= 8) {
            cudaEvent_t e0, e1;
            TDAGW_CUDA(cudaEventCreate(&e0));
            TDAGW_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            for (int gcand : gcs)
                for (int kcand : kss)
                    for (int fcand = 1; fcand >= 0; --fcand) {
                        run(gcand, kcand, fcand, 2, false);  // warm
                        TDAGW_CUDA(cudaEventRecord(e0, s));
                        run(gcand, kcand, fcand, 6, false);
                        TDAGW_CUDA(cudaEventRecord(e1, s));
                        TDAGW_CUDA(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        TDAGW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        if (ms < best) {
                            best = ms;
                            gc_max = gcand;
                            ks_max = kcand;
                            flags_on = fcand;
                        }
                    }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            int err = 0;
            TDAGW_CUDA(cudaMemcpy(&err, c.sync.as<unsigned>() + 2, sizeof(int), cudaMemcpyDeviceToHost));
            TDAGW_REQUIRE(!err, TDAGW_ERR_TIMEOUT, "a bounded wait gave up while tuning the tensor-core kernel");
            // the tuning runs overwrote the observables: restore the first row
            reset_batch_observables(c, bs, B);
            c.batch_plans[key] = {gc_max, ks_max | (flags_on << 20)};
        }
    }
    c.adj.valid = false;
    if (ckpt) {
        a.ckS = c.ckS.as<float2>();
        a.ckC = c.ckC.as<float2>();
        a.ck_period = period;
    }
    if (test_timeout) {
        a.extra_arrivals = 1;
        a.wait_ns = 20000000ull;
    }
    run(gc_max, ks_max, flags_on, bs.Tmax, !(flags & TDAGW_FLAG_NO_GRAPH) && !test_timeout);
    a.extra_arrivals = 0;
    a.wait_ns = 2000000000ull;
    c.persistent_launched = true;
    if (ckpt) {
        // the backward sweep: FP32 partition and arguments; segment recomputes on the
        // tensor cores from the checkpoints, with this launch's arguments
        prepare_adjoint_fp32(c, bs, fields, B, steps, dt, flags);
        AdjointState& st = c.adj;
        st.period = period;
        st.tc = true;
        a.ckS = nullptr;
        a.ckC = nullptr;
        st.tc_args.resize(sizeof(TcArgs));
        std::memcpy(st.tc_args.data(), &a, sizeof(TcArgs));
        st.tc_fn = fn;
        st.tc_smem = smem;
        st.tc_grid = nctas;
    }
    finish_batch(c, bs, B);
}

// Segment recompute of the adjoint's backward sweep (see the declaration): the checkpointed
// launch's arguments with the segment's first step and length, records on, checkpoints off,
// observables into scratch, the first stage's scales from the restored state, no resets.
void tc_recompute_segment(Ctx& c, int n0, int len, float2* recX, float2* recDS, double* obs) {
    AdjointState& st = c.adj;
    TDAGW_REQUIRE(st.valid && st.tc && st.tc_args.size() == sizeof(TcArgs), TDAGW_ERR_INVALID_ARG,
                  "no checkpointed tensor-core propagation to recompute");
    cudaStream_t s = c.stream;
    TcArgs a;
    std::memcpy(&a, st.tc_args.data(), sizeof(TcArgs));
    a.n0 = n0;
    a.Tmax = len;
    a.ckS = nullptr;
    a.ckC = nullptr;
    a.recX = recX;
    a.recDS = recDS;
    a.obs = obs;
    TDAGW_CUDA(cudaMemsetAsync(a.xmax, 0, 3 * (size_t)a.Bp * sizeof(unsigned), s));
    xmax_kernel<<<dim3(64, (unsigned)a.Bp), 256, 0, s>>>(a.X, a.N, a.Bp, a.xmax);
    check_launch("xmax_kernel");
    TDAGW_CUDA(cudaMemsetAsync(a.tdone, 0, (size_t)a.Nt * sizeof(unsigned long long), s));
    xtile_kernel<<<dim3((unsigned)a.Nt, (unsigned)a.Bp), 256, 0, s>>>(a.X, a.N, a.Bp, a.xtile);
    check_launch("xtile_kernel");
    TDAGW_CUDA(cudaMemsetAsync(c.sync.p, 0, 4 * sizeof(unsigned), s));
    void* args[] = {&a};
    TDAGW_CUDA(cudaLaunchCooperativeKernel(st.tc_fn, dim3(st.tc_grid), dim3(kTcThreads), args, st.tc_smem, s));
    c.persistent_launched = true;
}


// Split-FP16 tiles of the channel-wise factors (Eq. svd-channel-wise): V segment q as
// Mt_q = ceil(ldv_q / 256) column tiles x ceil(Nk / 16) chunks of k-points, U segment p
// (its low-rank columns, then the dense diagonal channel K^pp) as ceil(Nk / 256) row tiles
// x ceil(ldw_p / 16) chunks; power-of-two scales from the largest entries; the bound of
// the U-pass operand z_p = [S o y ; x_p]; the padded S o Y row of every gathered channel
// column.  Made once per set of channel factors.
void pack_channel_tc(Ctx& c) {
    ChannelFactors& f = c.ch;
    if (f.tc_valid) return;
    TDAGW_REQUIRE(c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED, "split-FP16 factors need a complex64 context");
    TDAGW_REQUIRE(f.valid, TDAGW_ERR_NO_FACTORS, "no channel factors installed");
    cudaStream_t s = c.stream;
    const ChMeta& m = f.m;
    const int P = m.P, Nk = m.Nk;
    const int nchK = (Nk + 15) / 16, NtK = (Nk + kRows - 1) / kRows;
    int maxc = 1;
    for (int e = 0; e < P; ++e) maxc = std::max(maxc, std::max(m.ldv[e], m.ldw[e]));
    DevBuf stats;
    stats.ensure((size_t)3 * maxc * sizeof(float));
    std::vector<float> st(3 * (size_t)maxc);
    float mu = 0.f, mv = 0.f, nv = 0.f, smax = 0.f;
    auto seg_stats = [&](const float2* A, int cols, bool isv) {
        factor_stats_kernel<<<(cols + 127) / 128, 128, 0, s>>>(A, A, Nk, cols, cols, stats.as<float>());
        check_launch("factor_stats_kernel");
        TDAGW_CUDA(cudaMemcpyAsync(st.data(), stats.p, 3 * (size_t)cols * sizeof(float), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
        for (int j = 0; j < cols; ++j) {
            if (isv) {
                mv = std::max(mv, st[j]);
                nv = std::max(nv, st[2 * (size_t)cols + j]);
            } else {
                mu = std::max(mu, st[j]);
            }
        }
    };
    f.tc_mtq0.assign(P + 1, 0);
    f.tc_nchw.assign(P, 0);
    f.tc_tvoff.assign(P, 0);
    f.tc_tuoff.assign(P, 0);
    long long tv = 0, tu = 0;
    for (int q = 0; q < P; ++q) {
        const int mt = (m.ldv[q] + kRows - 1) / kRows;
        f.tc_mtq0[q + 1] = f.tc_mtq0[q] + mt;
        f.tc_tvoff[q] = tv;
        tv += (long long)mt * nchK;
        if (m.ldv[q] > 0) seg_stats(f.V.as<float2>() + m.vbase[q], m.ldv[q], true);
    }
    for (int p = 0; p < P; ++p) {
        f.tc_nchw[p] = (m.ldw[p] + 15) / 16;
        f.tc_tuoff[p] = tu;
        tu += (long long)NtK * f.tc_nchw[p];
        seg_stats(f.U.as<float2>() + m.ubase[p], m.ldw[p], false);
    }
    std::vector<float> S((size_t)std::max<long long>(m.stot, 1), 0.f);
    if (m.stot > 0) {
        TDAGW_CUDA(cudaMemcpyAsync(S.data(), f.S.p, m.stot * sizeof(float), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
    for (float v : S) smax = std::max(smax, std::fabs(v));
    TDAGW_REQUIRE(std::isfinite(mu) && std::isfinite(mv) && std::isfinite(nv) && std::isfinite(smax),
                  TDAGW_ERR_INVALID_ARG, "factors are not finite");
    auto p2 = [](float bound) {
        if (!(bound > 0.f)) return 1.f;
        int e = 0;
        std::frexp(bound, &e);
        return std::ldexp(1.f, 13 - std::max(e, -100));
    };
    f.tc_su = p2(mu);
    f.tc_sv = p2(mv);
    // |y_c| <= ||v_c|| ||x_q|| <= ||v_c|| sqrt(2 Nk) max|x| for the channel columns, and
    // z_p also holds x_p itself
    f.tc_zbound = std::max(1.f, smax * std::sqrt(nv) * (float)std::sqrt(2.0 * (double)Nk));
    f.tcV.ensure((size_t)std::max<long long>(tv, 1) * kTile);
    f.tcU.ensure((size_t)std::max<long long>(tu, 1) * kTile);
    for (int q = 0; q < P; ++q) {
        if (m.ldv[q] == 0) continue;
        const int rp = (f.tc_mtq0[q + 1] - f.tc_mtq0[q]) * kRows;
        const int64_t total = (int64_t)nchK * 16 * rp;
        pack_v_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
            f.V.as<float2>() + m.vbase[q], Nk, m.ldv[q], m.ldv[q], rp, nchK, f.tc_sv,
            f.tcV.as<unsigned char>() + f.tc_tvoff[q] * kTile, total);
        check_launch("pack_v_kernel");
    }
    for (int p = 0; p < P; ++p) {
        const int rp = f.tc_nchw[p] * 16;
        const int64_t total = (int64_t)NtK * kRows * rp;
        pack_u_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
            f.U.as<float2>() + m.ubase[p], Nk, m.ldw[p], m.ldw[p], rp, f.tc_nchw[p], f.tc_su,
            f.tcU.as<unsigned char>() + f.tc_tuoff[p] * kTile, total);
        check_launch("pack_u_kernel");
    }
    // padded S o Y row of each gathered column (its V segment's tiles start at mtq0 256)
    std::vector<int> gpad((size_t)std::max<long long>(m.gtot, 1), 0);
    for (long long e = 0; e < m.gtot; ++e) {
        const long long col = f.gidx_host[e];
        int q = 0;
        while (q + 1 < P && m.sbase[q + 1] <= col) ++q;
        gpad[e] = f.tc_mtq0[q] * kRows + (int)(col - m.sbase[q]);
    }
    f.tcGpad.ensure(gpad.size() * sizeof(int));
    TDAGW_CUDA(cudaMemcpyAsync(f.tcGpad.p, gpad.data(), gpad.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    f.tcZero.ensure((size_t)c.hm.N * sizeof(float2));
    TDAGW_CUDA(cudaMemsetAsync(f.tcZero.p, 0, (size_t)c.hm.N * sizeof(float2), s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
    f.tc_valid = true;
}

void propagate_channel_tc(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt, int flags) {
    TDAGW_REQUIRE(c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED, "split-FP16 propagation needs a complex64 context");
    TDAGW_REQUIRE(flags & TDAGW_FLAG_RESET, TDAGW_ERR_UNSUPPORTED,
                  "split-FP16 propagation starts from drho = 0 (TDAGW_FLAG_RESET)");
    TDAGW_REQUIRE(!(flags & TDAGW_FLAG_CHECKPOINT), TDAGW_ERR_UNSUPPORTED,
                  "the channel-wise kernel runs without checkpoints");
    pack_channel_tc(c);
    const ChannelFactors& f = c.ch;
    const ChMeta& m = f.m;
    const HostModel& h = c.hm;
    cudaStream_t s = c.stream;
    const int64_t N = h.N;
    const int P = m.P, Nk = m.Nk;
    const int nchK = (Nk + 15) / 16, NtK = (Nk + kRows - 1) / kRows;
    const int nsegA = f.tc_mtq0[P];
    const int rp = std::max(1, nsegA) * kRows;
    const int nte = (int)((N + kRows - 1) / kRows);
    const BatchSetup bs = prepare_batch(c, fields, B, steps, dt);
    const int Bp = bs.Bp;

    int dev = 0, nsm = 0;
    TDAGW_CUDA(cudaGetDevice(&dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = tc_smem_bytes();
    const void* fn = h.Nb == 2 ? (const void*)batched_tc_kernel<2, true> : (const void*)batched_tc_kernel<4, true>;
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, smem));
    TDAGW_REQUIRE(per_sm == 1, TDAGW_ERR_UNSUPPORTED, "tensor-core batched kernel needs exactly one CTA per SM");
    const int nctas = nsm;

    const int KSmax = std::max(1, std::min(nctas / std::max(1, nsegA), nchK));
    c.tcP.ensure((size_t)KSmax * rp * Bp * sizeof(float2));
    c.tcY.ensure((size_t)rp * Bp * sizeof(float2));
    c.tcMax.ensure((size_t)3 * Bp * sizeof(unsigned));
    c.tcRed.ensure((size_t)4 * nte * Bp * 3 * sizeof(double));
    const size_t sbytes = (size_t)N * Bp * sizeof(float2);
    constexpr int kKcMax = 4;  // K-ranges of a phase C tile at most (partial dSigma slots)
    c.bdS.ensure(kKcMax * sbytes);
    c.sync.ensure(4 * sizeof(unsigned));

    TcArgs a{};
    a.tU = f.tcU.as<unsigned char>();
    a.tV = f.tcV.as<unsigned char>();
    a.Ys = c.tcY.as<float2>();
    a.P = c.tcP.as<float2>();
    a.xmax = c.tcMax.as<unsigned>();
    a.S = f.S.as<float>();
    a.diag = f.tcZero.as<float2>();  // the diagonal channels are products of phase C
    a.dx = c.dx.as<float2>();
    a.dy = c.dy.as<float2>();
    a.vx = c.vx.as<float2>();
    a.gap = c.gap.as<float2>();
    a.X = c.bX.as<float2>();
    a.Ssum = c.bS.as<float2>();
    a.Ccomp = c.bC.as<float2>();
    a.acc = c.bA.as<float2>();
    a.Etab = c.bEtab.as<double>();
    a.dir = c.bdir.as<float2>();
    a.act = c.bact.as<int>();
    a.red = c.tcRed.as<double>();
    a.obs = c.bobs.as<double>();
    a.bar = reinterpret_cast<unsigned long long*>(c.sync.p);
    a.err = reinterpret_cast<int*>(c.sync.as<unsigned>() + 2);
    a.N = N;
    a.ldE = bs.ldE;
    a.Nk = Nk;
    a.r = rp;
    a.rp = rp;
    a.Nt = P * NtK;  // phase C items per trajectory group
    a.Mt = nsegA;    // phase A column tiles per K-range
    a.nchU = 0;
    a.nchV = nchK;
    a.Bp = Bp;
    a.B = B;
    a.kahan = (flags & TDAGW_FLAG_NO_KAHAN) ? 0 : 1;
    a.c1 = h.c1;
    for (int q = 0; q < 4; ++q) a.occ[q] = (float)h.occ[q];
    a.dt = (float)dt;
    a.su = f.tc_su;
    a.sv = f.tc_sv;
    a.ybound = 0.f;
    a.wait_ns = 2000000000ull;
    a.n0 = 0;
    a.ck_period = 1;
    a.Nred = 4 * nte;  // per-quarter observable sums
    a.gpad = f.tcGpad.as<int>();
    a.dS = c.bdS.as<float2>();
    a.npair = P;
    a.NtK = NtK;
    a.nte = nte;
    a.zbound = f.tc_zbound;
    for (int e = 0; e < P; ++e) {
        a.tvoff[e] = f.tc_tvoff[e];
        a.tuoff[e] = f.tc_tuoff[e];
        a.mtq0[e] = f.tc_mtq0[e];
        a.ldvq[e] = m.ldv[e];
        a.sbq[e] = (int)m.sbase[e];
        a.nlrq[e] = m.nlr[e];
        a.gbq[e] = (int)m.gbase[e];
        a.nchw[e] = f.tc_nchw[e];
    }
    a.mtq0[P] = f.tc_mtq0[P];
    auto run = [&](int gc_max, int kc, int T, bool graph) {
        a.gc_max = gc_max;
        a.ks_max = 0;
        a.kcu = kc;
        a.Tmax = T;
        launch_batched(c, fn, dim3(nctas), dim3(kTcThreads), smem, &a, sizeof(a),
                       {{c.bX.p, sbytes},
                        {c.bS.p, sbytes},
                        {c.bC.p, sbytes},
                        {c.tcMax.p, 3 * Bp * sizeof(unsigned)},
                        {c.sync.p, 4 * sizeof(unsigned)}},
                       graph);
    };
    // work split tuned once per (B, channel columns) by timing six steps of each candidate:
    // the trajectory groups of phase C (as for the low-rank kernel) and the K-ranges of a
    // phase C tile (more ranges spread the U segments' tiles over more CTAs, at the cost of
    // partial dSigma sums in the epilogue)
    const uint64_t key = (0xF1ull << 56) | ((uint64_t)B << 32) | (uint64_t)(uint32_t)m.stot;
    int gc_max = 0, kc = 1;
    const bool test_timeout = (flags & TDAGW_FLAG_TEST_TIMEOUT) != 0;
    auto it = c.batch_plans.find(key);
    if (test_timeout) {
        // timeout test: no tuning; the launch below waits for an arrival that never comes
    } else if (it != c.batch_plans.end()) {
        gc_max = it->second.first;
        kc = it->second.second;
    } else {
        const int g_min = (B + kGroup - 1) / kGroup;
        const int g_fill = group_count(B, a.Nt, nctas, 0);
        std::vector<int> gcs;
        for (int gcand = g_min; gcand < g_fill; gcand *= 2) gcs.push_back(gcand);
        gcs.push_back(0);
        std::vector<int> kcs;
        for (int kcand = 1; kcand <= kKcMax; ++kcand) kcs.push_back(kcand);
        if (bs.Tmax >= 8) {
            cudaEvent_t e0, e1;
            TDAGW_CUDA(cudaEventCreate(&e0));
            TDAGW_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            for (int gcand : gcs)
                for (int kcand : kcs) {
                    run(gcand, kcand, 2, false);  // warm
                    TDAGW_CUDA(cudaEventRecord(e0, s));
                    run(gcand, kcand, 6, false);
                    TDAGW_CUDA(cudaEventRecord(e1, s));
                    TDAGW_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    TDAGW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) {
                        best = ms;
                        gc_max = gcand;
                        kc = kcand;
                    }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            int err = 0;
            TDAGW_CUDA(cudaMemcpy(&err, c.sync.as<unsigned>() + 2, sizeof(int), cudaMemcpyDeviceToHost));
            TDAGW_REQUIRE(!err, TDAGW_ERR_TIMEOUT, "a bounded wait gave up while tuning the tensor-core kernel");
            reset_batch_observables(c, bs, B);
            c.batch_plans[key] = {gc_max, kc};
        }
    }
    c.adj.valid = false;
    if (test_timeout) {
        a.extra_arrivals = 1;
        a.wait_ns = 20000000ull;
    }
    run(gc_max, kc, bs.Tmax, !(flags & TDAGW_FLAG_NO_GRAPH) && !test_timeout);
    c.persistent_launched = true;
    finish_batch(c, bs, B);
}

}  // namespace tdagw
