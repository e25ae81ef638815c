// Batched low-rank TD-aGW propagation on the fifth-generation tensor cores, with the
// truncated-SVD factors of Eq. svd_acc stored as split FP16 pairs (hi + lo, 8 bytes per
// complex element like complex64).
//
// Per RK4 stage the two products of the low-rank contraction,
//   Y = V^H X  (r x B)   and   dSigma = K^diag o X + U (S o Y)  (N x B),
// run as real tcgen05 kind::f16 MMAs with FP32 accumulation in tensor memory.  Complex
// arithmetic: the factor (the large, streamed operand) is read as an interleaved real
// matrix (re, im per complex column) and the small operand is expanded to 2 x 2 real
// blocks, so one real product yields real and imaginary parts in adjacent accumulator
// columns.  Split FP16: with a = s (a_hi + a_lo), each product is accumulated as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs; the dropped a_lo b_lo is 2^-22 relative).
// Power-of-two scales keep the FP16 values in range: 2^(13 - e) with 2^e above the largest
// magnitude, for U and V (measured once when the tiles are made) and, per trajectory, for
// X (the exact maximum of the stage input) and for S o Y (bound
// max|S| max_j ||v_j|| sqrt(2N) max|X|).
//
// Work of one stage (one cooperative launch for the whole propagation, one CTA per SM):
//   A  partials of V^H X over K-ranges of rows: CTA items (trajectory group, pair of
//      128-row tiles of V^H, K-range).  The V^H tiles (pre-tiled 16 KB blocks in the MMA's
//      shared-memory layout) stream through a ring by bulk copies; the expanded split X
//      block is built in shared memory by the worker warps.
//   -- grid barrier --
//   B  Y = S o sum of partials (fixed order), expanded and split into the B-operand tiles
//      of the second product.
//   -- grid barrier --
//   C  items (one or two 128-row tiles of U, trajectory group): U tiles and the Y tiles
//      they share stream through the ring; each accumulator (128 rows x 2 columns per
//      trajectory) is staged through shared memory in two halves and the commutator + RK4
//      epilogue (Eq. tdagw) runs per (k, b) block.
//   -- grid barrier --
// Roles: warp 0 streams tiles into the ring (running ahead across items), warp 1 issues
// the MMAs into one of two tensor-memory accumulators, warps 2-9 build operands and drain
// the other accumulator (epilogue of item i overlaps the MMAs of item i + 1).  Every wait
// is bounded; on expiry the kernel records an error, lets its own copies and MMAs finish
// (bounded waits), frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
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
// ring depth and built-B buffers (build-time tuning parameters; smem: (ring + buffers) x 16 KB)
#ifndef TDAGW_TC_RING
#define TDAGW_TC_RING 11
#endif
#ifndef TDAGW_TC_BBUF
#define TDAGW_TC_BBUF 2
#endif
constexpr int kRing = TDAGW_TC_RING;       // ring slots of one tile each
constexpr int kBBuf = TDAGW_TC_BBUF;       // built B blocks in flight (phase A)
static_assert(kRing + kBBuf <= 13, "ring and B buffers must fit in shared memory");
#ifndef TDAGW_TC_ATILES
#define TDAGW_TC_ATILES 4
#endif
// 128-row V^H tiles per phase A item (2: one accumulator buffer; 4: both buffers, i.e. two
// accumulator uses per item)
constexpr int kAMc = TDAGW_TC_ATILES;
static_assert(kAMc == 2 || kAMc == 4, "phase A items hold 2 or 4 V^H tiles");
constexpr int kCmb = 16;                   // chunk-completion barriers (ring); every wait on
                                           // one targets a chunk < kCmb chunks behind the
                                           // MMA thread's next chunk, so parities cannot alias
constexpr uint32_t kTile = 16384;          // 128 rows x 32 real columns, hi (8 KB) + lo (8 KB)
constexpr uint32_t kHalf = 8192;
constexpr int kKc = 32;                    // real reduction columns per tile (16 complex)
constexpr int kGroup = 64;                 // trajectories per group: MMA N = 2 x 64 max
constexpr uint32_t kLbo = 128, kSbo = (kKc / 8) * 128;
constexpr uint32_t kXbuf = kBBuf * kTile;  // B blocks (phase A) / staged half tile (phase C)
constexpr int kAccCols = 256;              // columns of one accumulator buffer (two buffers)
constexpr int kTmemCols = 512;

// staged half tile: 64 rows x 64 trajectories of float2, columns XOR-swizzled by row so
// that both the row-wise writes and the trajectory-wise reads avoid bank conflicts
__device__ __forceinline__ int ds_index(int row, int bl) {
    return row * 64 + (bl ^ (row & 31));
}

struct TcArgs {
    const unsigned char* tU;  // Nt x nchU tiles of U (rows) x 2r (real columns)
    const unsigned char* tV;  // Mt x nchV tiles of V^T (rows j) x 2 Np (real columns)
    unsigned char* tY;        // Gmax x nchU tiles: expanded split S o Y (rows 2b + c)
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
    double* red;  // Ntp x Bp x 3 (per phase C row-tile item)
    double* obs;  // (Tmax + 1) x B x 3
    unsigned long long* bar;
    int* err;
    int64_t N, ldE;
    int Nk, r, rp, Nt, Ntp, tpi, Mt, nchU, nchV, Bp, B, Tmax, kahan, c1;  // tpi: U row tiles per phase C item
    float occ[4];
    float dt;
    float su, sv;   // power-of-two scales of the U and V tiles
    float ybound;   // max|S| max_j ||v_j|| sqrt(2N): |(S o Y)_jb| <= ybound max|X_b|
    unsigned long long wait_ns;
};

// Optional phase timestamps (build with -DTDAGW_TRACE): one thread per CTA and role records
// %globaltimer at the phase boundaries of stages kTraceFirst .. kTraceFirst + kTraceStages - 1
// (points 0-6: stage start, end of A items, after barrier 1, end of B, after barrier 2, end
// of C items, after barrier 3; 7: MMA thread done with C items; 8: producer done with C
// tiles).
#ifdef TDAGW_TRACE
constexpr int kTraceFirst = 40, kTraceStages = 16;
__device__ unsigned long long g_trace_tc[160 * kTraceStages * 9];
#define TC_TRACE(who, k)                                                                         \
    do {                                                                                         \
        const int ts_ = 4 * n + st - kTraceFirst;                                                \
        if ((who) && blockIdx.x < 160 && ts_ >= 0 && ts_ < kTraceStages)                         \
            g_trace_tc[(blockIdx.x * kTraceStages + ts_) * 9 + (k)] = gtimer();                   \
    } while (0)
// per-chunk timestamps of phase A in CTA 0, stage kTraceFirst + 1, first item:
// [chunk][0] MMA thread has the chunk's tiles and B block, [1] its MMAs are issued,
// [2] worker 0 may overwrite the B buffer, [3] worker 0 has built the block;
// [63][0..3]: worker 0 accumulator ready, readout done, MMA thread item done, -
__device__ unsigned long long g_trace_a[64 * 4];
#define TC_TRACE_A(who, cc, k)                                                                   \
    do {                                                                                         \
        if ((who) && blockIdx.x == 0 && 4 * n + st == kTraceFirst + 1 && item == (int)blockIdx.x && (cc) < 64) \
            g_trace_a[(cc) * 4 + (k)] = gtimer();                                                 \
    } while (0)
// wait/issue time accumulators per CTA and traced stage: [0] MMA thread waiting for tiles,
// [1] for B blocks, [2] for a free accumulator, [3] issuing MMAs and commits, [4] copy
// thread waiting for a free slot, [5] issuing copies
__device__ unsigned long long g_trace_w[160 * kTraceStages * 6];
#define TC_W_BEGIN(id) const uint64_t tw_##id = gtimer()
#define TC_W_END(id, k)                                                                          \
    do {                                                                                         \
        const int ts_ = 4 * n + st - kTraceFirst;                                                \
        if (blockIdx.x < 160 && ts_ >= 0 && ts_ < kTraceStages)                                  \
            g_trace_w[(blockIdx.x * kTraceStages + ts_) * 6 + (k)] += gtimer() - tw_##id;         \
    } while (0)
#else
#define TC_TRACE(who, k) \
    do {                 \
    } while (0)
#define TC_TRACE_A(who, cc, k) \
    do {                       \
    } while (0)
#define TC_W_BEGIN(id) \
    do {               \
    } while (0)
#define TC_W_END(id, k) \
    do {                \
    } while (0)
#endif

// non-blocking test (copy and MMA threads poll) and potentially blocking test (workers:
// the hardware may suspend the thread until the phase completes)
__device__ __forceinline__ bool mb_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc::smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
#ifndef TDAGW_TC_WORKER_POLL
#define TDAGW_TC_WORKER_POLL 0  // 1: worker warps poll (test_wait) instead of try_wait
#endif
// bounded wait for the phase of the given parity; false on expiry or abort
template <bool POLL>
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, volatile int* abort_s,
                                        unsigned long long budget) {
    if (POLL ? mb_test(b, parity) : mbar_try(b, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (POLL ? mb_test(b, parity) : mbar_try(b, parity)) return true;
        if ((i & 63) == 0) {
            if (abort_s && *abort_s) return false;
            if (gtimer() - t0 > budget) return false;
        }
    }
}
#ifndef TDAGW_TC_EVICT_FIRST
#define TDAGW_TC_EVICT_FIRST 1  // factor tiles are streamed with an L2 evict-first policy
#endif
__device__ __forceinline__ void workers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory");
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

// grid barrier over the monotonic arrival counter (all threads call)
__device__ bool tc_grid_sync(const TcArgs& a, unsigned& gen, int* abort_s) {
    __syncthreads();
    if (threadIdx.x == 0 && !*abort_s) {
        const unsigned long long target = (unsigned long long)(gen + 1) * gridDim.x;
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
        gen += 1;
    }
    __syncthreads();
    return !*(volatile int*)abort_s;
}

// the three split products of one 128 x N x 32 tile pair (two K = 16 steps each)
__device__ __forceinline__ void mma_tile(uint32_t d, uint32_t a_addr, uint32_t b_addr, uint32_t idesc, bool first) {
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ah = tc::sdesc(a_addr + ks * 256, kLbo, kSbo);
        const uint64_t al = tc::sdesc(a_addr + kHalf + ks * 256, kLbo, kSbo);
        const uint64_t bh = tc::sdesc(b_addr + ks * 256, kLbo, kSbo);
        const uint64_t bl = tc::sdesc(b_addr + kHalf + ks * 256, kLbo, kSbo);
        tc::mma_f16(d, ah, bh, idesc, (first && ks == 0) ? 0u : 1u);
        tc::mma_f16(d, ah, bl, idesc, 1u);
        tc::mma_f16(d, al, bh, idesc, 1u);
    }
}

// Commutator + RK4 stage update of one (k, trajectory) block (Eq. tdagw; the arithmetic of
// the FP32 batched path), with the low-rank part of dSigma read from the staged half tile
// (block rows row0 .. row0 + NB^2 - 1, trajectory column bl) and K^diag o X added here.
// xm: running max(|Re|, |Im|) of the values written to X (the next stage input).
template <int NB>
__device__ Obs3 stage_kb_tc(const TcArgs& a, int k, int b, int st, float E, float2 dr,
                            const float2* sDS, int row0, int bl, float& xm) {
    constexpr int NB2 = NB * NB;
    const int64_t Bp = a.Bp;
    float2 X[NB2], M[NB2];
#pragma unroll
    for (int g = 0; g < NB2; ++g) {
        const int64_t i = (int64_t)k * NB2 + g;
        X[g] = __ldcg(a.X + i * Bp + b);
        const float2 d1 = a.dx[i], d2 = a.dy[i];
        const float2 ds = cfma(a.diag[i], X[g], sDS[ds_index(row0 + g, bl)]);
        M[g] = make_float2(ds.x + E * (dr.x * d1.x + dr.y * d2.x), ds.y + E * (dr.x * d1.y + dr.y * d2.y));
    }
    Obs3 ob{0.0, 0.0, 0.0};
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
                ob.p += (double)rho.x * (double)d1.x + (double)rho.y * (double)d1.y;
                ob.j += (double)rho.x * (double)v1.x + (double)rho.y * (double)v1.y;
                if (n == m && n == a.c1) ob.o += (double)rho.x;
            }
            a.X[e] = Xn;
            xm = fmaxf(xm, fmaxf(fabsf(Xn.x), fabsf(Xn.y)));
        }
    }
    return ob;
}

// Trajectory groups: at most kGroup trajectories each, and enough groups for about one
// item of the U product per CTA (row tiles x groups <= CTAs) while groups keep >= 8.
__host__ __device__ __forceinline__ int group_count(int Bact, int Nt, int nctas) {
    const int g_min = (Bact + kGroup - 1) / kGroup;
    const int g_fill = min(max(1, nctas / Nt), (Bact + 7) / 8);
    return max(g_min, g_fill);
}
struct Groups {
    int G, MGn, KS;  // phase A: trajectory groups, groups of kAMc V^H tiles, K-ranges
    int GC;          // phase C (and B): trajectory groups
};
__device__ __forceinline__ Groups stage_groups(const TcArgs& a, int Bact) {
    Groups q;
    q.G = group_count(Bact, a.Nt, (int)gridDim.x);
    q.GC = group_count(Bact, a.Ntp, (int)gridDim.x);
    q.MGn = (a.Mt + kAMc - 1) / kAMc;
    q.KS = max(1, min((int)gridDim.x / max(1, q.G * q.MGn), a.nchV));
    return q;
}
// phase A item -> (trajectory group, first V^H tile, tile count, chunk range)
struct ItemA {
    int g, m0, mc, ks, c0, c1;
};
__device__ __forceinline__ ItemA item_a(const TcArgs& a, const Groups& q, int item) {
    ItemA it;
    it.g = item % q.G;
    const int mg = (item / q.G) % q.MGn;
    it.ks = item / (q.G * q.MGn);
    it.m0 = kAMc * mg;
    it.mc = min(kAMc, a.Mt - it.m0);
    it.c0 = (int)((int64_t)it.ks * a.nchV / q.KS);
    it.c1 = (int)((int64_t)(it.ks + 1) * a.nchV / q.KS);
    return it;
}

template <int NB>
__global__ void __launch_bounds__(kTcThreads, 1) batched_tc_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ring = smem;
    unsigned char* xbuf = ring + kRing * kTile;
    float2* sDS = reinterpret_cast<float2*>(xbuf);
    double* sred = reinterpret_cast<double*>(xbuf + kXbuf);
    float* ssc = reinterpret_cast<float*>(sred + kWorkers * 3);
    unsigned* smx = reinterpret_cast<unsigned*>(ssc + kGroup);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smx + kGroup);
    uint64_t* full = bars;
    uint64_t* cmb = full + kRing;     // MMAs of chunk q complete (one commit per chunk)
    uint64_t* bfull = cmb + kCmb;
    uint64_t* accf = bfull + kBBuf;   // accumulator written (MMA -> workers)
    uint64_t* acce = accf + 2;    // accumulator drained (workers -> MMA)
    uint64_t* fin = acce + 2;     // last MMAs complete (teardown)
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = tid == 0, mma = tid == 32, worker = warp >= 2;
    const int wt = tid - 64;  // worker index
    constexpr int NB2 = NB * NB;
    const unsigned long long budget = a.wait_ns;
    volatile int* vabort = &abort_s;

    if (tid == 0) {
        abort_s = 0;
        for (int s = 0; s < kRing; ++s) mbar_init(full + s, 1);
        for (int s = 0; s < kCmb; ++s) mbar_init(cmb + s, 1);
        for (int s = 0; s < kBBuf; ++s) mbar_init(bfull + s, kWorkers);
        for (int s = 0; s < 2; ++s) {
            mbar_init(accf + s, 1);
            mbar_init(acce + s, kWorkers);
        }
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
    uint32_t bu = 0;    // uses of the built-B buffers (MMA thread and workers)
    uint32_t acnt = 0;  // uses of the two accumulators (MMA thread and workers)
    int gch = 0;        // chunks so far (all roles count the same sequence)
    int slot_ch[kRing]; // producer: chunk that last used each ring slot
    int buf_ch[kBBuf];  // workers: chunk that last used each B buffer
    for (int q = 0; q < kRing; ++q) slot_ch[q] = -1;
    for (int q = 0; q < kBBuf; ++q) buf_ch[q] = -1;
    unsigned gen = 0;
    bool ok = true;
    auto fail = [&]() {
        atomicExch(a.err, 1);
        abort_s = 1;
    };
    // wait until the MMAs of chunk q are complete (q < 0: nothing to wait for; a chunk
    // kCmb or more behind is complete: an accumulator wait or a grid barrier came between)
    auto chunk_done = [&](int q, bool poll) -> bool {
        if (q < 0 || gch - q >= kCmb) return true;
        return poll ? mb_wait<true>(cmb + q % kCmb, (uint32_t)(q / kCmb) & 1u, vabort, budget)
                    : mb_wait<TDAGW_TC_WORKER_POLL != 0>(cmb + q % kCmb, (uint32_t)(q / kCmb) & 1u, vabort, budget);
    };
    const uint64_t ef_policy = TDAGW_TC_EVICT_FIRST ? policy_evict_first() : 0ull;
    // producer: one tile of chunk gch into the next ring slot (factor tiles may carry an
    // evict-first L2 policy)
    auto issue = [&](const unsigned char* src, bool factor) {
        if (*vabort) return;
        const uint32_t slot = ppos % kRing;
        if (!chunk_done(slot_ch[slot], true)) {
            fail();
            return;
        }
        slot_ch[slot] = gch;
        mbar_expect_tx(full + slot, kTile);
        if (TDAGW_TC_EVICT_FIRST && factor)
            bulk_g2s_hint(ring + slot * kTile, src, kTile, full + slot, ef_policy);
        else
            bulk_g2s(ring + slot * kTile, src, kTile, full + slot);
        ++ppos;
    };
    // MMA thread: wait for the next tile; returns its shared-memory address (0 on failure)
    auto next_tile = [&]() -> uint32_t {
        const uint32_t slot = mpos % kRing, use = mpos / kRing;
        if (*vabort || !mb_wait<true>(full + slot, use & 1u, vabort, budget)) {
            fail();
            return 0u;
        }
        ++mpos;
        return tc::smem_u32(ring + slot * kTile);
    };
    auto end_chunk = [&]() {  // MMA thread: the chunk's MMAs are issued
        tc::mma_commit(cmb + gch % kCmb);
    };

    for (int n = 0; n < a.Tmax && ok; ++n) {
        const int Bact = a.act[n];
        const Groups q = stage_groups(a, Bact);
        for (int st = 0; st < 4 && ok; ++st) {
            const int gs = 4 * n + st;
            const unsigned* xin = a.xmax + (gs % 3) * a.Bp;
            unsigned* xout = a.xmax + ((gs + 1) % 3) * a.Bp;
            TC_TRACE(producer, 0);
            if (blockIdx.x == 0 && worker)
                for (int b = wt; b < a.Bp; b += kWorkers) xout[b] = 0u;

            // ---------------- A: partials of V^H X ----------------
            const int nA = q.G * q.MGn * q.KS;
            if (producer) {
                for (int item = blockIdx.x; item < nA; item += gridDim.x) {
                    const ItemA it = item_a(a, q, item);
                    for (int c = it.c0; c < it.c1; ++c, ++gch) {
                        TC_W_BEGIN(p0);
                        for (int ml = 0; ml < it.mc; ++ml) issue(a.tV + ((int64_t)(it.m0 + ml) * a.nchV + c) * kTile, true);
                        TC_W_END(p0, 4);
                    }
                }
            } else if (mma) {
                for (int item = blockIdx.x; item < nA; item += gridDim.x) {
                    const ItemA it = item_a(a, q, item);
                    int b0, b1;
                    group_range(Bact, q.G, it.g, b0, b1);
                    const int nbp = (b1 - b0 + 7) & ~7;
                    const int nuse = (it.mc + 1) / 2;  // accumulator uses (two tiles each)
                    TC_W_BEGIN(a0);
                    for (int u = 0; u < nuse; ++u) {
                        const uint32_t k = acnt + u;
                        if (*vabort || !mb_wait<true>(acce + (k & 1u), ((k >> 1) & 1u) ^ 1u, vabort, budget)) fail();
                    }
                    TC_W_END(a0, 2);
                    tc::fence_after_sync();
                    const uint32_t idesc = tc::idesc_f16(128, 2 * nbp);
                    for (int c = it.c0; c < it.c1 && !*vabort; ++c) {
                        uint32_t ta[kAMc] = {};
                        TC_W_BEGIN(t0);
                        for (int ml = 0; ml < it.mc; ++ml) ta[ml] = next_tile();
                        TC_W_END(t0, 0);
                        TC_W_BEGIN(b0);
                        if (*vabort || !mb_wait<true>(bfull + bu % kBBuf, (bu / kBBuf) & 1u, vabort, budget)) {
                            fail();
                            break;
                        }
                        TC_W_END(b0, 1);
                        TC_TRACE_A(true, c - it.c0, 0);
                        tc::fence_after_sync();
                        const uint32_t baddr = tc::smem_u32(xbuf + (bu % kBBuf) * kTile);
                        TC_W_BEGIN(m0);
                        for (int ml = 0; ml < it.mc; ++ml)
                            mma_tile(tm + ((acnt + ml / 2) & 1u) * kAccCols + (ml % 2) * 128, ta[ml], baddr, idesc,
                                     c == it.c0);
                        TC_TRACE_A(true, c - it.c0, 1);
                        end_chunk();
                        TC_W_END(m0, 3);
                        ++gch;
                        ++bu;
                    }
                    for (int u = 0; u < nuse; ++u) tc::mma_commit(accf + ((acnt + u) & 1u));
                    TC_TRACE_A(true, 63, 2);
                    acnt += nuse;
                }
            } else if (worker) {
                for (int item = blockIdx.x; item < nA; item += gridDim.x) {
                    const ItemA it = item_a(a, q, item);
                    int b0, b1;
                    group_range(Bact, q.G, it.g, b0, b1);
                    const int nbg = b1 - b0, nbp = (nbg + 7) & ~7;
                    workers_sync();  // the previous item's readers of ssc are done
                    if (wt < kGroup) ssc[wt] = wt < nbg ? pow2_scale(__uint_as_float(__ldcg(xin + b0 + wt))) : 0.f;
                    workers_sync();
                    // expanded split X block of each chunk (16 rows x nbp trajectories); each
                    // worker owns elements e = wt + 256 u, u < 4, and loads the values of the
                    // chunk after next before building the current one
                    constexpr int kPer = 16 * kGroup / kWorkers;
                    auto load_chunk = [&](int c, float2 (&xv)[kPer]) {
#pragma unroll
                        for (int u = 0; u < kPer; ++u) {
                            const int e = wt + kWorkers * u;
                            const int il = (e & 3) | ((e >> 8) << 2), bl = (e >> 2) & 63;
                            const int64_t i = (int64_t)c * 16 + il;
                            xv[u] = (bl < nbg && i < a.N) ? __ldcg(a.X + i * a.Bp + b0 + bl) : make_float2(0.f, 0.f);
                        }
                    };
                    auto build_chunk = [&](int c, const float2 (&xv)[kPer]) {
                        const uint32_t bs = bu % kBBuf;
                        if (!*vabort && !chunk_done(buf_ch[bs], false)) fail();
                        buf_ch[bs] = gch;
                        TC_TRACE_A(wt == 0, c - it.c0, 2);
                        if (!*vabort) {
                            unsigned char* tile = xbuf + bs * kTile;
#pragma unroll
                            for (int u = 0; u < kPer; ++u) {
                                const int e = wt + kWorkers * u;
                                const int il = (e & 3) | ((e >> 8) << 2), bl = (e >> 2) & 63;
                                if (bl >= nbp) continue;
                                const float2 x = xv[u];
                                const float sx = ssc[bl];
                                __half rh, rl, ih, il2;
                                split16(x.x * sx, rh, rl);
                                split16(x.y * sx, ih, il2);
                                const uint32_t o0 = tc::kmajor_offset(2 * bl, 2 * il, kKc);
                                const uint32_t o1 = tc::kmajor_offset(2 * bl + 1, 2 * il, kKc);
                                *reinterpret_cast<__half2*>(tile + o0) = __halves2half2(rh, ih);
                                *reinterpret_cast<__half2*>(tile + o1) = __halves2half2(ih, __hneg(rh));
                                *reinterpret_cast<__half2*>(tile + kHalf + o0) = __halves2half2(rl, il2);
                                *reinterpret_cast<__half2*>(tile + kHalf + o1) = __halves2half2(il2, __hneg(rl));
                            }
                        }
                        tc::fence_proxy_async();
                        mbar_arrive(bfull + bs);
                        TC_TRACE_A(wt == 0, c - it.c0, 3);
                        ++bu;
                        ++gch;
                    };
                    // expanded split X block of each chunk (16 rows x nbp trajectories); each
                    // worker owns elements e = wt + 256 u, u < 4; its loads run two chunks
                    // ahead of the build (three rotating register sets, no copies)
                    float2 xa[kPer], xb[kPer], xc[kPer];
                    if (it.c0 < it.c1) load_chunk(it.c0, xa);
                    if (it.c0 + 1 < it.c1) load_chunk(it.c0 + 1, xb);
                    for (int c = it.c0; c < it.c1; c += 3) {
                        if (c + 2 < it.c1) load_chunk(c + 2, xc);
                        build_chunk(c, xa);
                        if (c + 1 >= it.c1) break;
                        if (c + 3 < it.c1) load_chunk(c + 3, xa);
                        build_chunk(c + 1, xb);
                        if (c + 2 >= it.c1) break;
                        if (c + 4 < it.c1) load_chunk(c + 4, xb);
                        build_chunk(c + 2, xc);
                    }
                    // accumulators -> raw partials P[ks][j][b], 64 rows at a time staged in
                    // the (now idle) B buffers so that the global writes run along
                    // trajectories (coalesced)
                    const int nuse = (it.mc + 1) / 2;
                    for (int u = 0; u < nuse; ++u) {
                        const uint32_t k = acnt + u;
                        if (!*vabort && !mb_wait<TDAGW_TC_WORKER_POLL != 0>(accf + (k & 1u), (k >> 1) & 1u, vabort, budget))
                            fail();
                    }
                    TC_TRACE_A(wt == 0, 63, 0);
                    tc::fence_after_sync();
                    float2* stg = reinterpret_cast<float2*>(xbuf);  // 64 rows x 64 float2 (32 KB)
                    const int quarter = warp & 3, half = (warp - 2) >> 2;
                    const int units = (2 * nbp) / 16, uh = (units + 1) / 2;
                    for (int ml = 0; ml < it.mc; ++ml) {
                        TC_TRACE_A(wt == 0, 62, ml);
                        for (int ph = 0; ph < 2; ++ph) {
                            workers_sync();  // B buffers / the previous half no longer read
                            if ((quarter >> 1) == ph && !*vabort) {
                                const int row = 32 * (quarter & 1) + lane;
                                for (int u = half * uh; u < min(units, (half + 1) * uh); ++u) {
                                    float v[16];
                                    tc::tmem_ld16(tm + ((uint32_t)(32 * quarter) << 16) + ((acnt + ml / 2) & 1u) * kAccCols +
                                                      (ml % 2) * 128 + 16 * u,
                                                  v);
#pragma unroll
                                    for (int p = 0; p < 8; ++p)
                                        stg[ds_index(row, 8 * u + p)] = make_float2(v[2 * p], v[2 * p + 1]);
                                }
                            }
                            workers_sync();
                            if (!*vabort) {
                                float2* pbase = a.P + ((int64_t)it.ks * a.rp + (it.m0 + ml) * 128 + 64 * ph) * a.Bp + b0;
                                for (int e = wt; e < 64 * nbg; e += kWorkers) {
                                    const int row = e / nbg, bl = e % nbg;
                                    pbase[(int64_t)row * a.Bp + bl] = stg[ds_index(row, bl)];
                                }
                            }
                        }
                    }
                    workers_sync();  // staging reads done before the next item's B blocks
                    tc::fence_before_sync();
                    for (int u = 0; u < nuse; ++u) mbar_arrive(acce + ((acnt + u) & 1u));
                    TC_TRACE_A(wt == 0, 63, 1);
                    acnt += nuse;
                }
            }
            TC_TRACE(producer, 1);
            if (!(ok = tc_grid_sync(a, gen, &abort_s))) break;
            TC_TRACE(producer, 2);

            // ---------------- B: Y = S o sum of partials -> split expanded tiles ----------------
            {
                const int64_t gt = (int64_t)blockIdx.x * kTcThreads + tid, total = (int64_t)gridDim.x * kTcThreads;
                // elements (g, j, bl) of all groups, flattened
                int64_t tot_el = 0;
                for (int g = 0; g < q.GC; ++g) {
                    int b0, b1;
                    group_range(Bact, q.GC, g, b0, b1);
                    tot_el += (int64_t)a.rp * ((b1 - b0 + 7) & ~7);
                }
                for (int64_t e = gt; e < tot_el; e += total) {
                    int g = 0, b0 = 0, b1 = 0, nbp = 0;
                    int64_t rem = e;
                    for (;; ++g) {
                        group_range(Bact, q.GC, g, b0, b1);
                        nbp = (b1 - b0 + 7) & ~7;
                        const int64_t sz = (int64_t)a.rp * nbp;
                        if (rem < sz || g == q.GC - 1) break;
                        rem -= sz;
                    }
                    const int nbg = b1 - b0;
                    const int j = (int)(rem / nbp), bl = (int)(rem % nbp);
                    float2 v = make_float2(0.f, 0.f);
                    if (bl < nbg && j < a.r) {
                        const int b = b0 + bl;
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
                        const float sx = pow2_scale(mx), sy = pow2_scale(a.ybound * mx);
                        v = cscale(s, a.S[j] * (sy / (a.sv * sx)));
                    }
                    __half rh, rl, ih, il;
                    split16(v.x, rh, rl);
                    split16(v.y, ih, il);
                    unsigned char* tile = a.tY + ((int64_t)g * a.nchU + j / 16) * kTile;
                    const uint32_t o0 = tc::kmajor_offset(2 * bl, 2 * (j % 16), kKc);
                    const uint32_t o1 = tc::kmajor_offset(2 * bl + 1, 2 * (j % 16), kKc);
                    *reinterpret_cast<__half2*>(tile + o0) = __halves2half2(rh, __hneg(ih));
                    *reinterpret_cast<__half2*>(tile + o1) = __halves2half2(ih, rh);
                    *reinterpret_cast<__half2*>(tile + kHalf + o0) = __halves2half2(rl, __hneg(il));
                    *reinterpret_cast<__half2*>(tile + kHalf + o1) = __halves2half2(il, rl);
                }
                if (st == 0 && n > 0) {
                    // observables of step n (written by the last stage of step n - 1)
                    for (int64_t b = gt; b < a.act[n - 1]; b += total) {
                        double s0 = 0, s1 = 0, s2 = 0;
                        for (int t = 0; t < a.Ntp; ++t) {
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
            // the tiles were written through the generic proxy and are read by bulk copies
            asm volatile("fence.proxy.async;" ::: "memory");
            TC_TRACE(producer, 3);
            if (!(ok = tc_grid_sync(a, gen, &abort_s))) break;
            TC_TRACE(producer, 4);

            // ---------------- C: dSigma = U (S o Y) + K^diag o X, commutator, RK4 ----------------
            const int eoff = st == 0 ? 0 : (st == 3 ? 2 : 1);
            const int nC = a.Ntp * q.GC;
            if (producer) {
                for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                    const int t0 = a.tpi * (item % a.Ntp), g = item / a.Ntp;
                    const int tcnt = min(a.tpi, a.Nt - t0);
                    for (int c = 0; c < a.nchU; ++c, ++gch) {
                        TC_W_BEGIN(p1);
                        for (int u = 0; u < tcnt; ++u) issue(a.tU + ((int64_t)(t0 + u) * a.nchU + c) * kTile, true);
                        issue(a.tY + ((int64_t)g * a.nchU + c) * kTile, false);
                        TC_W_END(p1, 4);
                    }
                }
                TC_TRACE(true, 8);
            } else if (mma) {
                for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                    const int t0 = a.tpi * (item % a.Ntp), g = item / a.Ntp;
                    const int tcnt = min(a.tpi, a.Nt - t0);
                    int b0, b1;
                    group_range(Bact, q.GC, g, b0, b1);
                    const int nbp = (b1 - b0 + 7) & ~7;
                    const uint32_t ab = acnt & 1u;
                    TC_W_BEGIN(a0);
                    if (*vabort || !mb_wait<true>(acce + ab, ((acnt >> 1) & 1u) ^ 1u, vabort, budget)) fail();
                    TC_W_END(a0, 2);
                    tc::fence_after_sync();
                    const uint32_t idesc = tc::idesc_f16(128, 2 * nbp);
                    for (int c = 0; c < a.nchU && !*vabort; ++c) {
                        uint32_t tu[2] = {0u, 0u};
                        TC_W_BEGIN(t1);
                        for (int u = 0; u < tcnt; ++u) tu[u] = next_tile();
                        const uint32_t ty = next_tile();
                        TC_W_END(t1, 0);
                        if (*vabort) break;
                        tc::fence_after_sync();
                        TC_W_BEGIN(m1);
                        for (int u = 0; u < tcnt; ++u) mma_tile(tm + ab * kAccCols + u * 128, tu[u], ty, idesc, c == 0);
                        end_chunk();
                        TC_W_END(m1, 3);
                        ++gch;
                    }
                    tc::mma_commit(accf + ab);
                    ++acnt;
                }
                TC_TRACE(true, 7);
            } else if (worker) {
                for (int item = blockIdx.x; item < nC; item += gridDim.x) {
                    const int tp = item % a.Ntp, t0 = a.tpi * tp, g = item / a.Ntp;
                    const int tcnt = min(a.tpi, a.Nt - t0);
                    gch += a.nchU;  // the item's chunks (counted like the copy and MMA threads)
                    int b0, b1;
                    group_range(Bact, q.GC, g, b0, b1);
                    const int nbg = b1 - b0, nbp = (nbg + 7) & ~7;
                    workers_sync();  // the previous item's readers of ssc, smx, sred are done
                    if (wt < kGroup) {
                        if (wt < nbg) {
                            const float mx = __uint_as_float(__ldcg(xin + b0 + wt));
                            ssc[wt] = 1.f / (a.su * pow2_scale(a.ybound * mx));
                        }
                        smx[wt] = 0u;
                    }
                    workers_sync();
                    const uint32_t ab = acnt & 1u;
                    if (!*vabort && !mb_wait<TDAGW_TC_WORKER_POLL != 0>(accf + ab, (acnt >> 1) & 1u, vabort, budget)) fail();
                    tc::fence_after_sync();
                    const int quarter = warp & 3, half = (warp - 2) >> 2;
                    const int units = (2 * nbp) / 16, uh = (units + 1) / 2;
                    const int kgroups = kWorkers / nbg;
                    const int bl = wt % nbg, kg = wt / nbg;
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                    float xm = 0.f;
                    for (int u2 = 0; u2 < a.tpi; ++u2) {
                        const int t = t0 + u2;
                        for (int ph = 0; ph < 2; ++ph) {
                            // accumulator rows 64 ph .. +63 (lane quarters 2 ph, 2 ph + 1) -> staged half
                            if (u2 < tcnt && (quarter >> 1) == ph && !*vabort) {
                                const int row = 32 * (quarter & 1) + lane;
                                for (int u = half * uh; u < min(units, (half + 1) * uh); ++u) {
                                    float v[16];
                                    tc::tmem_ld16(tm + ((uint32_t)(32 * quarter) << 16) + ab * kAccCols + u2 * 128 + 16 * u, v);
#pragma unroll
                                    for (int p = 0; p < 8; ++p) {
                                        const int b2 = 8 * u + p;
                                        if (b2 < nbg)
                                            sDS[ds_index(row, b2)] = make_float2(v[2 * p] * ssc[b2], v[2 * p + 1] * ssc[b2]);
                                    }
                                }
                            }
                            workers_sync();
                            // commutator + RK4 for the k-blocks of these 64 rows
                            const int kbase = (t * 128 + 64 * ph) / NB2;
                            const int kt = u2 < tcnt ? min(64 / NB2, a.Nk - kbase) : 0;
                            if (kg < kgroups && !*vabort) {
                                const int b = b0 + bl;
                                const float E = (float)a.Etab[(int64_t)b * a.ldE + 2 * n + eoff];
                                const float2 dr = a.dir[b];
                                for (int kl = kg; kl < kt; kl += kgroups) {
                                    const Obs3 ob = stage_kb_tc<NB>(a, kbase + kl, b, st, E, dr, sDS, kl * NB2, bl, xm);
                                    s0 += ob.p;
                                    s1 += ob.j;
                                    s2 += ob.o;
                                }
                            }
                            workers_sync();  // the staged half is consumed before it is rewritten
                        }
                    }
                    tc::fence_before_sync();
                    mbar_arrive(acce + ab);
                    ++acnt;
                    if (kg < kgroups) {
                        atomicMax(smx + bl, __float_as_uint(xm));
                        if (st == 3) {
                            sred[(kg * nbg + bl) * 3] = s0;
                            sred[(kg * nbg + bl) * 3 + 1] = s1;
                            sred[(kg * nbg + bl) * 3 + 2] = s2;
                        }
                    }
                    workers_sync();
                    if (wt < nbg && !*vabort) {
                        atomicMax(xout + b0 + wt, smx[wt]);
                        if (st == 3) {
                            double r0 = 0.0, r1 = 0.0, r2 = 0.0;
                            for (int k2 = 0; k2 < kgroups; ++k2) {
                                r0 += sred[(k2 * nbg + wt) * 3];
                                r1 += sred[(k2 * nbg + wt) * 3 + 1];
                                r2 += sred[(k2 * nbg + wt) * 3 + 2];
                            }
                            double* rr = a.red + ((int64_t)tp * a.Bp + b0 + wt) * 3;
                            rr[0] = r0;
                            rr[1] = r1;
                            rr[2] = r2;
                        }
                    }
                }
            }
            TC_TRACE(producer, 5);
            ok = tc_grid_sync(a, gen, &abort_s);
            TC_TRACE(producer, 6);
        }
    }
    // observables of the last step
    if (ok && a.Tmax > 0) {
        const int n = a.Tmax;
        const int64_t gt = (int64_t)blockIdx.x * kTcThreads + tid, total = (int64_t)gridDim.x * kTcThreads;
        for (int64_t b = gt; b < a.act[n - 1]; b += total) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int t = 0; t < a.Ntp; ++t) {
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
        for (uint32_t p = first; p < ppos; ++p) mb_wait<true>(full + p % kRing, (p / kRing) & 1u, nullptr, budget);
    }
    if (mma) {
        tc::mma_commit(fin);
        mb_wait<true>(fin, 0u, nullptr, budget);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, kTmemCols);
    }
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

// Split-FP16 tiles of U: tile (t, c) holds rows 128 t .. +127 and complex columns
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
    unsigned char* tile = out + ((i / 128) * nchU + j / 16) * (int64_t)kTile;
    const uint32_t o = tc::kmajor_offset((uint32_t)(i % 128), 2 * (j % 16), kKc);
    *reinterpret_cast<__half2*>(tile + o) = __halves2half2(rh, ih);
    *reinterpret_cast<__half2*>(tile + kHalf + o) = __halves2half2(rl, il);
}

// Split-FP16 tiles of V^T: tile (m, c) holds rows j = 128 m .. +127 (columns of V) and
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
    unsigned char* tile = out + ((int64_t)(j / 128) * nchV + i / 16) * (int64_t)kTile;
    const uint32_t o = tc::kmajor_offset((uint32_t)(j % 128), (uint32_t)(2 * (i % 16)), kKc);
    *reinterpret_cast<__half2*>(tile + o) = __halves2half2(rh, ih);
    *reinterpret_cast<__half2*>(tile + kHalf + o) = __halves2half2(rl, il);
}

struct TcDims {
    int Nt, Np, rp, Mt, nchU, nchV;
};
TcDims tc_dims(int64_t N, int r) {
    TcDims d;
    d.Nt = (int)((N + 127) / 128);
    d.Np = d.Nt * 128;
    d.rp = (r + 127) / 128 * 128;
    d.Mt = d.rp / 128;
    d.nchU = 2 * d.rp / kKc;
    d.nchV = 2 * d.Np / kKc;
    return d;
}

size_t tc_smem_bytes() {
    return (size_t)kRing * kTile + kXbuf + (size_t)kWorkers * 3 * sizeof(double) + kGroup * sizeof(float) +
           kGroup * sizeof(unsigned) + (kRing + kCmb + kBBuf + 5) * sizeof(uint64_t);
}

}  // namespace

#ifdef TDAGW_TRACE
extern "C" int tdagw_debug_trace_tc(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_trace_tc, sizeof(unsigned long long) * (size_t)n) == cudaSuccess ? 0 : -3;
}
extern "C" int tdagw_debug_trace_tc_w(unsigned long long* out) {
    return cudaMemcpyFromSymbol(out, g_trace_w, sizeof(unsigned long long) * 160 * kTraceStages * 6) == cudaSuccess ? 0 : -3;
}
extern "C" int tdagw_debug_trace_tc_a(unsigned long long* out) {
    return cudaMemcpyFromSymbol(out, g_trace_a, sizeof(unsigned long long) * 64 * 4) == cudaSuccess ? 0 : -3;
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
    TDAGW_REQUIRE(!(flags & TDAGW_FLAG_CHECKPOINT), TDAGW_ERR_UNSUPPORTED,
                  "checkpoints for the adjoint are kept by the FP32 path only");
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
    const void* fn = h.Nb == 2 ? (const void*)batched_tc_kernel<2> : (const void*)batched_tc_kernel<4>;
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, smem));
    TDAGW_REQUIRE(per_sm == 1, TDAGW_ERR_UNSUPPORTED, "tensor-core batched kernel needs exactly one CTA per SM");
    const int nctas = nsm;

    // largest split of the V^H X reduction over the run (one trajectory group)
    const int MGn = (d.Mt + 3) / 4;
    const int KSmax = std::max(1, std::min(nctas / MGn, d.nchV));
    // two U row tiles per phase C item (sharing the S o Y tiles) only when each CTA has
    // several items: the epilogue of a CTA's last item is not overlapped by MMAs
    int tpi = d.Nt >= 4 * nctas ? 2 : 1;
    if (const char* e = std::getenv("TDAGW_TC_TILES_PER_ITEM")) {  // tuning override (1 or 2)
        const int v = std::atoi(e);
        if (v == 1 || v == 2) tpi = v;
    }
    const int Ntp = (d.Nt + tpi - 1) / tpi;
    const int Gmax = group_count(B, Ntp, nctas);
    c.tcP.ensure((size_t)KSmax * d.rp * Bp * sizeof(float2));
    c.tcY.ensure((size_t)Gmax * d.nchU * kTile);
    c.tcMax.ensure((size_t)3 * Bp * sizeof(unsigned));
    c.tcRed.ensure((size_t)Ntp * Bp * 3 * sizeof(double));
    const size_t sbytes = (size_t)N * Bp * sizeof(float2);
    c.sync.ensure(4 * sizeof(unsigned));

    TcArgs a{};
    a.tU = c.tcU.as<unsigned char>();
    a.tV = c.tcV.as<unsigned char>();
    a.tY = c.tcY.as<unsigned char>();
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
    a.N = N;
    a.ldE = bs.ldE;
    a.Nk = h.Nk;
    a.r = r;
    a.rp = d.rp;
    a.Nt = d.Nt;
    a.Ntp = Ntp;
    a.tpi = tpi;
    a.Mt = d.Mt;
    a.nchU = d.nchU;
    a.nchV = d.nchV;
    a.Bp = Bp;
    a.B = B;
    a.Tmax = bs.Tmax;
    a.kahan = (flags & TDAGW_FLAG_NO_KAHAN) ? 0 : 1;
    a.c1 = h.c1;
    for (int q = 0; q < 4; ++q) a.occ[q] = (float)h.occ[q];
    a.dt = (float)dt;
    a.su = c.tc_su;
    a.sv = c.tc_sv;
    a.ybound = c.tc_ybound;
    a.wait_ns = 2000000000ull;
    launch_batched(c, fn, dim3(nctas), dim3(kTcThreads), smem, &a, sizeof(a),
                   {{c.bX.p, sbytes},
                    {c.bS.p, sbytes},
                    {c.bC.p, sbytes},
                    {c.tcMax.p, 3 * Bp * sizeof(unsigned)},
                    {c.sync.p, 4 * sizeof(unsigned)}},
                   !(flags & TDAGW_FLAG_NO_GRAPH));
    c.persistent_launched = true;
    c.adj.valid = false;
    finish_batch(c, bs, B);
}

}  // namespace tdagw
