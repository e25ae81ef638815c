// Persistent channel-wise TD-aGW propagation (single trajectory, complex64): one
// cooperative launch runs all RK4 steps of a call with the kernel in the channel-wise form
// of Eq. svd-channel-wise (dense diagonal channels, truncated SVDs of the off-diagonal
// channels).  Per stage:
//
//   V pass   for each input pair q:  y_c = sum_{k' of this CTA} conj(V_q[k']) x[k' P + q]
//   grid barrier; x by pair (Xt[p][k]) from this CTA's rows; S o sum_c y_c (column slice)
//   grid barrier; U pass  for the rows (p, k) of this CTA's share of the U segments:
//            dSigma[k P + p] = U_p[k] . [S o y of the channels out of p ; x_p]
//   grid barrier; commutator, RK4 stage update, observables for the CTA's own k
//
// Each CTA owns a contiguous range of k-points with all their pair elements: its V pass
// reads only its own stage input and its commutators write it, so no barrier separates
// them.  The U pass instead splits the stacked U segments (rows (p, k), p-major, one
// contiguous array) into byte-balanced contiguous shares: a CTA streams one range of
// rows touching one or two pairs (two vectors z_p instead of all P), and the dSigma rows
// reach their k-point's owner through L2 across a third barrier.  The dense diagonal
// channels need all of x_p: every CTA publishes its rows of the stage input by pair after
// the first barrier (when no CTA still reads the previous stage's), and reads x_p after
// the second.  A producer warp streams the CTA's V rows and its U share through a
// shared-memory ring with 1D bulk copies (L2 evict-first: the factors are read once per
// stage), sixteen consumer warps compute from shared memory.
// Every wait is bounded; on expiry the CTA records an error word and returns.
#include <algorithm>

#include "common.cuh"
#include "persist.cuh"
#include "stage.cuh"

namespace tdagw {

namespace {

using namespace persist;

constexpr int kCW = 16;              // consumer warps
constexpr int kCons = kCW * 32;
constexpr int kThr = kCons + 32;
constexpr int kSlotMin = 32768;      // bytes per ring slot (at least one whole row) ...
constexpr int kSlotMax = 65536;      // ... up to four U rows when those are long
constexpr int kZPre = 8;             // U-pass vector entries prefetched per thread (<= 4096)

// Optional phase timestamps (build with -DTDAGW_TRACE): thread 0 of every CTA records
// %globaltimer at nine points of each of the first kChTraceStages stages, and when its
// waits for the first V-pass slots return (points 9 ...).
#ifdef TDAGW_TRACE
constexpr int kChTraceStages = 16;
constexpr int kChTracePts = 16;
__device__ unsigned long long g_trace_ch[160 * kChTraceStages * kChTracePts];
#define CH_TRACE(k)                                                                         \
    do {                                                                                    \
        if (tid == 0 && cta < 160 && n * 4 + st < kChTraceStages && (k) < kChTracePts)      \
            g_trace_ch[(cta * kChTraceStages + n * 4 + st) * kChTracePts + (k)] = gtimer(); \
    } while (0)
#else
#define CH_TRACE(k) \
    do {            \
    } while (0)
#endif

struct CHArgs {
    ChMeta m;
    const float2* V;
    const float2* U;
    const float* S;
    const int* gidx;
    StageParams<float> sp;
    float2* dSw;   // dSigma written by the U pass (sp.dS reads it)
    float2* part;  // gridDim x stot partial y vectors
    float2* ytil;  // stot, S o y
    float2* Xt;    // P x Nk, stage input by pair
    unsigned long long* bar_count;
    int* err;
    int T, nslots, slot_bytes, kmax, zs_len, upart_len;
    int vgroups;  // V pass: warp groups (power of two), each owning every vgroups-th pair
    int extra_arrivals;  // > 0 only for the timeout test: the barrier can never complete
    unsigned long long wait_ns;
};

// First U-pass row of CTA c (global row p Nk + k of the stacked U segments, which are
// contiguous and p-major): the first row that starts at or after c/G of the U elements,
// so that the shares are balanced to a row.
__host__ __device__ inline int urow_start(const ChMeta& m, int c, int G) {
    const long long t = (long long)c * m.utot / G;
    for (int p = 0; p < m.P; ++p) {
        const long long end = m.ubase[p] + (long long)m.Nk * m.ldw[p];
        if (t < end) {
            const long long k = (t - m.ubase[p] + m.ldw[p] - 1) / m.ldw[p];
            return p * m.Nk + (int)k;
        }
    }
    return m.P * m.Nk;
}

// rows of a segment per ring slot: the largest power of two (<= 64) whose rows fit
__device__ __forceinline__ int seg_rps(int ld, int slot_bytes) {
    int r = 1;
    while (r < 64 && 2 * r * ld * 8 <= slot_bytes) r *= 2;
    return r;
}

// The V pass streams its chunks (up to seg_rps rows of one input pair) packed into shared
// slots: consecutive chunks share a slot while they fit, so the short segments of the V
// pass still fill the ring.  VWalk is the walk over those chunks that the producer and
// the consumers both follow; qi counts the non-empty pairs passed (the pair's owner group
// in the consumers is qi mod the number of groups).
struct VWalk {
    int q, r0, qi;
    __device__ __forceinline__ void skip_empty(const ChMeta& m, int P) {
        while (q < P && m.ldv[q] == 0) ++q;
    }
    // bytes of the current chunk and its row count
    __device__ __forceinline__ uint32_t chunk(const ChMeta& m, int nk, int slot_bytes, int& nr) const {
        const int ld = m.ldv[q];
        nr = min(seg_rps(ld, slot_bytes), nk - r0);
        return (uint32_t)nr * ld * 8u;
    }
    __device__ __forceinline__ void next(const ChMeta& m, int P, int nk, int nr) {
        r0 += nr;
        if (r0 >= nk) {
            r0 = 0;
            ++q;
            ++qi;
            skip_empty(m, P);
        }
    }
};

template <int NB>
__global__ void __launch_bounds__(kThr, 1) ch_persistent_kernel(CHArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int P = NB * NB;
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int Nk = a.m.Nk;
    const int ka = (int)((int64_t)cta * Nk / G), kb = (int)((int64_t)(cta + 1) * Nk / G);
    const int nk = kb - ka;
    const int64_t ra = (int64_t)ka * P, rb = (int64_t)kb * P;
    const int ns = a.nslots;
    // this CTA's share of the U pass: rows [ur0, ur1) of the stacked U segments, pairs
    // pA .. pB (pB < pA when the share is empty)
    const int ur0 = urow_start(a.m, cta, G), ur1 = urow_start(a.m, cta + 1, G);
    const int pA = ur0 / Nk, pB = ur1 > ur0 ? (ur1 - 1) / Nk : pA - 1;

    unsigned char* ring = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)ns * a.slot_bytes);
    uint64_t* empty = full + ns;
    float2* zbuf = reinterpret_cast<float2*>(empty + ns);  // 2 x zs_len U-pass vectors
    float2* ubuf = zbuf + 2 * a.zs_len;                    // 2 x upart_len partial dots
    float2* xs = ubuf + 2 * a.upart_len;                   // kmax x P, this CTA's stage input
    float2* yred = xs + a.kmax * P;                         // kCons partial sums of S o y
    double* wred = reinterpret_cast<double*>(yred + kCons);
    volatile int* abort_s = reinterpret_cast<volatile int*>(wred + 3 * kCW);

    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kCW);
        }
        *abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kCW) {
        // ------------------------------------------------------------ producer warp
        if (lane == 0) {
            RingPos pos{0, 0u};
            uint64_t issued = 0;
            bool ok = true;
            const uint64_t policy = policy_evict_first();
            for (int n = 0; n < a.T && ok; ++n)
                for (int st = 0; st < 4 && ok; ++st) {
                    // V pass: chunks of consecutive input pairs packed into shared slots
                    VWalk vw{0, 0, 0};
                    vw.skip_empty(a.m, P);
                    while (vw.q < P) {
                        if (issued >= (uint64_t)ns &&
                            !mbar_wait(empty + pos.slot, pos.phase ^ 1u, abort_s, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        VWalk end = vw;
                        uint32_t tot = 0;
                        while (end.q < P) {
                            int nr;
                            const uint32_t b = end.chunk(a.m, nk, a.slot_bytes, nr);
                            if (tot > 0 && tot + b > (uint32_t)a.slot_bytes) break;
                            tot += b;
                            end.next(a.m, P, nk, nr);
                        }
                        mbar_expect_tx(full + pos.slot, tot);
                        uint32_t off = 0;
                        while (vw.q != end.q || vw.r0 != end.r0) {
                            int nr;
                            const uint32_t b = vw.chunk(a.m, nk, a.slot_bytes, nr);
                            const int ld = a.m.ldv[vw.q];
                            bulk_g2s_hint(ring + (size_t)pos.slot * a.slot_bytes + off,
                                          a.V + a.m.vbase[vw.q] + (int64_t)(ka + vw.r0) * ld, b, full + pos.slot,
                                          policy);
                            off += b;
                            vw.next(a.m, P, nk, nr);
                        }
                        ++issued;
                        pos.advance(1, ns);
                    }
                    // U pass: this CTA's share, one chunk of rows of one pair per slot
                    for (int e = pA; e <= pB && ok; ++e) {
                        const int ld = a.m.ldw[e];
                        const int k0 = e == pA ? ur0 - pA * Nk : 0, k1 = e == pB ? ur1 - pB * Nk : Nk;
                        const int nkp = k1 - k0;
                        const float2* base = a.U + a.m.ubase[e] + (int64_t)k0 * ld;
                        const int rps = seg_rps(ld, a.slot_bytes);
                        for (int r0 = 0; r0 < nkp; r0 += rps) {
                            if (issued >= (uint64_t)ns &&
                                !mbar_wait(empty + pos.slot, pos.phase ^ 1u, abort_s, a.wait_ns)) {
                                ok = false;
                                break;
                            }
                            const int nr = min(rps, nkp - r0);
                            const uint32_t bytes = (uint32_t)nr * ld * 8u;
                            mbar_expect_tx(full + pos.slot, bytes);
                            bulk_g2s_hint(ring + (size_t)pos.slot * a.slot_bytes, base + (int64_t)r0 * ld, bytes,
                                          full + pos.slot, policy);
                            ++issued;
                            pos.advance(1, ns);
                        }
                    }
                }
            if (!ok) {
                atomicExch(a.err, 1);
                *abort_s = 1;
            }
            // every issued copy must land before the CTA may exit
            const int back = issued < (uint64_t)ns ? (int)issued : ns;
            for (int j = 1; j <= back; ++j) {
                int s2 = pos.slot - j;
                uint32_t ph = pos.phase;
                if (s2 < 0) {
                    s2 += ns;
                    ph ^= 1u;
                }
                mbar_wait(full + s2, ph, nullptr, a.wait_ns);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ consumer warps
        const int64_t stot = a.m.stot;
        const int j0 = (int)(cta * stot / G), j1 = (int)((cta + 1) * stot / G);
        const int nj = j1 - j0, nsub = nj > 0 ? kCons / nj : 0;  // nj <= 512: stot <= 16 x 2048
        unsigned lgen = 0;
        RingPos pos{0, 0u};
        bool ok = true;
        for (int e = tid; e < nk * P; e += kCons) xs[e] = __ldcg(a.sp.X + ra + e);
        named_sync<kCons>();
        for (int n = 0; n < a.T && ok; ++n) {
            for (int st = 0; st < 4 && ok; ++st) {
                CH_TRACE(0);
                // ---- V pass: the consumer warps form vgroups groups of TG threads; a pair's
                //      chunks all go to one group (pairs dealt round-robin), whose thread lt
                //      owns column pairs lt and lt + TG of the segment (ldv <= 4 TG), so the
                //      short V rows keep every warp busy; one slot may hold chunks of
                //      several consecutive pairs, every warp waits for and releases each slot
                {
                    const int wpg = kCW / a.vgroups, TG = 32 * wpg;
                    const int vg = warp / wpg, lt = tid - vg * TG;
                    VWalk vw{0, 0, 0};
                    vw.skip_empty(a.m, P);
                    float2 acc[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
                    int vslot = 0;
                    while (vw.q < P) {
                        if (!warp_wait_full(full, pos, abort_s, a.wait_ns, lane)) break;
                        CH_TRACE(9 + vslot);
                        ++vslot;
                        const unsigned char* sbase = ring + (size_t)pos.slot * a.slot_bytes;
                        uint32_t off = 0;
                        while (vw.q < P) {
                            int nr;
                            const uint32_t b = vw.chunk(a.m, nk, a.slot_bytes, nr);
                            if (off > 0 && off + b > (uint32_t)a.slot_bytes) break;
                            const int q = vw.q, ld = a.m.ldv[q];
                            const float2* tile = reinterpret_cast<const float2*>(sbase + off);
                            // other groups' pairs and warps without columns of this pair
                            // skip the rows; two rows per iteration
                            const bool own = (vw.qi & (a.vgroups - 1)) == vg;
                            if (own && 64 * (warp - vg * wpg) < ld) {
                                const float2* xr = xs + vw.r0 * P + q;
#pragma unroll
                                for (int m = 0; m < 2; ++m) {
                                    const int c = 2 * (lt + m * TG);
                                    if (c < ld) {
                                        float2 a0 = acc[2 * m], a1 = acc[2 * m + 1];
                                        float2 b0 = make_float2(0.f, 0.f), b1 = b0;
                                        int rr = 0;
                                        for (; rr + 1 < nr; rr += 2) {
                                            const float4 v = *reinterpret_cast<const float4*>(tile + (size_t)rr * ld + c);
                                            const float4 w = *reinterpret_cast<const float4*>(tile + (size_t)(rr + 1) * ld + c);
                                            const float2 x0 = xr[rr * P], x1 = xr[(rr + 1) * P];
                                            a0 = cfmac(make_float2(v.x, v.y), x0, a0);
                                            a1 = cfmac(make_float2(v.z, v.w), x0, a1);
                                            b0 = cfmac(make_float2(w.x, w.y), x1, b0);
                                            b1 = cfmac(make_float2(w.z, w.w), x1, b1);
                                        }
                                        if (rr < nr) {
                                            const float4 v = *reinterpret_cast<const float4*>(tile + (size_t)rr * ld + c);
                                            const float2 x0 = xr[rr * P];
                                            a0 = cfmac(make_float2(v.x, v.y), x0, a0);
                                            a1 = cfmac(make_float2(v.z, v.w), x0, a1);
                                        }
                                        acc[2 * m] = cadd(a0, b0);
                                        acc[2 * m + 1] = cadd(a1, b1);
                                    }
                                }
                            }
                            off += b;
                            if (own && vw.r0 + nr >= nk) {  // last chunk of pair q: publish its partials
                                float2* dst = a.part + (size_t)cta * stot + a.m.sbase[q];
#pragma unroll
                                for (int m = 0; m < 2; ++m) {
                                    const int p2 = lt + m * TG;
                                    if (2 * p2 < ld)
                                        *reinterpret_cast<float4*>(dst + 2 * p2) = make_float4(
                                            acc[2 * m].x, acc[2 * m].y, acc[2 * m + 1].x, acc[2 * m + 1].y);
                                }
#pragma unroll
                                for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
                            }
                            vw.next(a.m, P, nk, nr);
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(empty + pos.slot);
                        pos.advance(1, ns);
                    }
                }
                CH_TRACE(1);
                if (!(ok = grid_sync<kCons>(a.bar_count, a.err, a.extra_arrivals, a.wait_ns, lgen, abort_s))) break;
                CH_TRACE(2);
                // ---- every CTA has finished the previous stage: publish this stage's input
                //      by pair for the dense diagonal channels
                for (int e = tid; e < nk * P; e += kCons) {
                    const int kk = e / P, p = e % P;
                    a.Xt[(int64_t)p * Nk + ka + kk] = xs[e];
                }
                // observables of the previous step (all partials were published at its last
                // stage, before this barrier); the last warp is idle in the sums below
                if (st == 0 && n > 0 && cta == 0 && warp == kCW - 1)
                    reduce_obs_row(a.sp.red, G, 1.0 / (double)Nk, a.sp.obs + 3 * (int64_t)n, lane);
                // ---- S o sum_c y_c for this CTA's columns: thread = (column, subset of the
                //      partials), then the subsets in a fixed order
                if (nj > 0) {
                    const int sub = tid / nj, col = tid % nj;
                    if (sub < nsub) {
                        float2 s = make_float2(0.f, 0.f);
                        for (int c2 = sub; c2 < G; c2 += nsub) s = cadd(s, __ldcg(a.part + (size_t)c2 * stot + j0 + col));
                        yred[sub * nj + col] = s;
                    }
                    named_sync<kCons>();
                    if (tid < nj) {
                        float2 s = yred[tid];
                        for (int u = 1; u < nsub; ++u) s = cadd(s, yred[u * nj + tid]);
                        a.ytil[j0 + tid] = cscale(s, a.S[j0 + tid]);
                    }
                }
                CH_TRACE(3);
                if (!(ok = grid_sync<kCons>(a.bar_count, a.err, a.extra_arrivals, a.wait_ns, lgen, abort_s))) break;
                CH_TRACE(4);
                // ---- U pass, per output pair p: the rows of a tile are split over the
                //      consumer warps by column parts ((row in tile) x parts = 16 warps).
                //      The vector of pair p + 1 is loaded into registers while pair p's
                //      tiles are consumed (its S o y entries and x_{p+1} come from L2), and
                //      stored into the other buffer before the barrier that ends pair p.
                float2 zr[kZPre];
                auto zload = [&](int pp) {
                    const int nl = a.m.nlr[pp];
                    const int* g = a.gidx + a.m.gbase[pp];
#pragma unroll
                    for (int j = 0; j < kZPre; ++j) {
                        const int c = tid + j * kCons;
                        zr[j] = c < nl ? __ldcg(a.ytil + __ldg(g + c))
                                       : (c < nl + Nk ? __ldcg(a.Xt + (int64_t)pp * Nk + (c - nl))
                                                      : make_float2(0.f, 0.f));
                    }
                };
                auto zstore = [&](float2* dst, int ld) {
#pragma unroll
                    for (int j = 0; j < kZPre; ++j) {
                        const int c = tid + j * kCons;
                        if (c < ld) dst[c] = zr[j];
                    }
                };
                if (pA <= pB) {
                    zload(pA);
                    zstore(zbuf, a.m.ldw[pA]);
                }
                named_sync<kCons>();
                CH_TRACE(5);
                for (int p = pA; p <= pB; ++p) {
                    const int ld = a.m.ldw[p];
                    const int k0 = p == pA ? ur0 - pA * Nk : 0, k1 = p == pB ? ur1 - pB * Nk : Nk;
                    const int nkp = k1 - k0;
                    const float2* zs = zbuf + ((p - pA) & 1) * a.zs_len;
                    float2* upart = ubuf + ((p - pA) & 1) * a.upart_len;
                    if (p + 1 <= pB) zload(p + 1);
                    const int rps = seg_rps(ld, a.slot_bytes);
                    const int cp = rps >= kCW ? 1 : kCW / rps;
                    const int pw = ((ld + cp - 1) / cp + 1) / 2 * 2;
                    const int myq = warp % cp, myr = warp / cp, rstride = kCW / cp;
                    const int c0 = myq * pw, c1 = min(ld, c0 + pw);
                    for (int r0 = 0; r0 < nkp; r0 += rps) {
                        if (!warp_wait_full(full, pos, abort_s, a.wait_ns, lane)) break;
                        const float2* tile = reinterpret_cast<const float2*>(ring + (size_t)pos.slot * a.slot_bytes);
                        const int nr = min(rps, nkp - r0);
                        for (int rr = myr; rr < nr; rr += rstride) {
                            const float2* ur = tile + (size_t)rr * ld;
                            float2 d = make_float2(0.f, 0.f), d1 = d;
                            for (int col = c0 + 2 * lane; col < c1; col += 64) {
                                const float4 u = *reinterpret_cast<const float4*>(ur + col);
                                const float4 zv = *reinterpret_cast<const float4*>(zs + col);
                                d = cfma(make_float2(u.x, u.y), make_float2(zv.x, zv.y), d);
                                d1 = cfma(make_float2(u.z, u.w), make_float2(zv.z, zv.w), d1);
                            }
                            d = cadd(d, d1);
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) d = cadd(d, shfl_xor(d, o));
                            if (lane == 0) upart[(r0 + rr) * cp + myq] = d;
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(empty + pos.slot);
                        pos.advance(1, ns);
                    }
                    if (p + 1 <= pB) zstore(zbuf + ((p + 1 - pA) & 1) * a.zs_len, a.m.ldw[p + 1]);
                    // every part of every row of pair p is in, and the vector of p + 1; the
                    // buffers written next (pair p + 2) were last read before this barrier's
                    // predecessor
                    named_sync<kCons>();
                    for (int kk = tid; kk < nkp; kk += kCons) {
                        float2 s = upart[kk * cp];
                        for (int qq = 1; qq < cp; ++qq) s = cadd(s, upart[kk * cp + qq]);
                        a.dSw[(int64_t)(k0 + kk) * P + p] = s;
                    }
                }
                // every CTA's dSigma rows are complete (the own k-points' rows came from
                // the CTAs whose U shares hold them)
                if (!(ok = grid_sync<kCons>(a.bar_count, a.err, a.extra_arrivals, a.wait_ns, lgen, abort_s))) break;
                CH_TRACE(6);
                // ---- commutator + RK4 stage update for k in [ka, kb)
                const int eoff = st == 0 ? 0 : (st == 3 ? 2 : 1);
                const float E = (float)a.sp.Etab[2 * (int64_t)n + eoff];
                ObsDF ob;  // double-float sums (FP64 is slow on this GPU)
                for (int64_t b = ra; b < rb; b += kCons) {
                    const int64_t i = b + tid;
                    stage_element<float, NB>(a.sp, i, i < rb, lane, st, E, ob);
                }
                if (st == 3) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        ob.p = ob.p.shfl_xor_sum(o);
                        ob.j = ob.j.shfl_xor_sum(o);
                        ob.o = ob.o.shfl_xor_sum(o);
                    }
                    float* wf = reinterpret_cast<float*>(wred);  // 6 floats per warp
                    if (lane == 0) {
                        wf[6 * warp] = ob.p.hi;
                        wf[6 * warp + 1] = ob.p.lo;
                        wf[6 * warp + 2] = ob.j.hi;
                        wf[6 * warp + 3] = ob.j.lo;
                        wf[6 * warp + 4] = ob.o.hi;
                        wf[6 * warp + 5] = ob.o.lo;
                    }
                    named_sync<kCons>();
                    if (tid == 0) {
                        ObsDF s;
                        for (int w = 0; w < kCW; ++w) {
                            DF t;
                            t.hi = wf[6 * w];
                            t.lo = wf[6 * w + 1];
                            s.p.add(t);
                            t.hi = wf[6 * w + 2];
                            t.lo = wf[6 * w + 3];
                            s.j.add(t);
                            t.hi = wf[6 * w + 4];
                            t.lo = wf[6 * w + 5];
                            s.o.add(t);
                        }
                        a.sp.red[3 * cta] = s.p.value();
                        a.sp.red[3 * cta + 1] = s.j.value();
                        a.sp.red[3 * cta + 2] = s.o.value();
                    }
                }
                CH_TRACE(7);
                for (int e = tid; e < nk * P; e += kCons) xs[e] = __ldcg(a.sp.X + ra + e);
                named_sync<kCons>();
                CH_TRACE(8);
            }
        }
        // observables of the last step: every CTA's partial is published by one more barrier
        if (ok && a.T > 0) {
            ok = grid_sync<kCons>(a.bar_count, a.err, a.extra_arrivals, a.wait_ns, lgen, abort_s);
            if (ok && cta == 0 && warp == 0)
                reduce_obs_row(a.sp.red, G, 1.0 / (double)Nk, a.sp.obs + 3 * (int64_t)a.T, lane);
        }
        // ok is uniform here: it only changes through grid_sync, which every consumer
        // thread enters in the same order and which returns the same shared flag to all
        if (!ok && tid == 0) {
            atomicExch(a.err, 1);
            *abort_s = 1;
        }
    }
    __syncthreads();
}

}  // namespace

#ifdef TDAGW_TRACE
extern "C" int tdagw_debug_trace_ch(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_trace_ch, sizeof(unsigned long long) * (size_t)n) == cudaSuccess ? 0 : -3;
}
#endif

// Host side: launch geometry, ring sizing, cooperative launch.  Returns false when the path
// does not apply (complex128, an input pair with more than 2048 low-rank columns, U rows
// longer than 4096 entries, too little shared memory); the caller then runs the stage-wise
// kernels.
bool launch_ch_persistent(Ctx& c, int T, double dt, double dirx, double diry, bool kahan,
                          bool test_timeout, cudaStream_t s) {
    const HostModel& h = c.hm;
    ChannelFactors& f = c.ch;
    const ChMeta& m = f.m;
    if (c.dtype != TDAGW_C64 || !f.valid) return false;
    const int P = h.Nb * h.Nb;
    int maxv = 0, maxw = 0;
    for (int e = 0; e < P; ++e) {
        maxv = std::max(maxv, m.ldv[e]);
        maxw = std::max(maxw, m.ldw[e]);
    }
    if (maxv > 4 * kCons) return false;  // V pass: two column pairs per consumer thread
    int dev = 0, nsm = 0, smem_max = 0, coop = 0;
    TDAGW_CUDA(cudaGetDevice(&dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return false;
    const int G = (int)std::min<int64_t>(nsm, h.Nk);  // every CTA owns >= 1 k-point
    const int kmax = (h.Nk + G - 1) / G;
    const int row_max = std::max(maxv, maxw) * 8;
    const int zs_len = maxw;  // even
    if (zs_len > kZPre * kCons) return false;  // the U-pass vector prefetch covers 4096 entries
    const size_t extras_fixed = 2 * (size_t)zs_len * 8 + (size_t)kmax * P * 8 + (size_t)kCons * 8 + 3 * kCW * 8 + 16;
    const size_t avail = (size_t)smem_max - 1024;
    // slots of up to four U rows (fewer partial dot products per row), as long as at least
    // four slots fit; at least one whole row
    auto slot_for = [&](int rows) {
        return (std::max(kSlotMin, std::max(row_max, std::min(rows * maxw * 8, kSlotMax))) + 127) / 128 * 128;
    };
    // partial dot products of one pair of a U share: rows x column parts (per slot size)
    auto upart_need = [&](int sb) {
        int need = 1;
        for (int c = 0; c < G; ++c) {
            const int u0 = urow_start(m, c, G), u1 = urow_start(m, c + 1, G);
            for (int p = u0 / h.Nk; u1 > u0 && p <= (u1 - 1) / h.Nk; ++p) {
                const int k0 = std::max(u0, p * h.Nk), k1 = std::min(u1, (p + 1) * h.Nk);
                int rps = 1;
                while (rps < 64 && 2 * rps * m.ldw[p] * 8 <= sb) rps *= 2;
                const int cp = rps >= kCW ? 1 : kCW / rps;
                need = std::max(need, (k1 - k0) * cp);
            }
        }
        return need;
    };
    int slot_bytes = 0, upart_len = 0;
    size_t extras = 0;
    for (int rows = 4; rows >= 1 && !slot_bytes; rows /= 2) {
        const int sb = slot_for(rows);
        const int ul = upart_need(sb);
        const size_t ex = extras_fixed + 2 * (size_t)ul * 8;
        if (avail > ex && (avail - ex) / ((size_t)sb + 16) >= 4) {
            slot_bytes = sb;
            upart_len = ul;
            extras = ex;
        }
    }
    if (!slot_bytes) return false;
    const int nslots = (int)std::min<size_t>(64, (avail - extras) / (slot_bytes + 16));
    const size_t smem = (size_t)nslots * slot_bytes + 16 * (size_t)nslots + extras;

    CHArgs a{};
    a.m = m;
    a.V = f.V.as<float2>();
    a.U = f.U.as<float2>();
    a.S = f.S.as<float>();
    a.gidx = f.gidx.as<int>();
    StageParams<float>& p = a.sp;
    p.X = c.X.as<float2>();
    p.dS = c.dS.as<float2>();
    p.dx = c.dx.as<float2>();
    p.dy = c.dy.as<float2>();
    p.vx = c.vx.as<float2>();
    p.gap = c.gap.as<float2>();
    p.acc = c.acc.as<float2>();
    p.Ssum = c.Ssum.as<float2>();
    p.Ccomp = c.Ccomp.as<float2>();
    p.Xnext = c.X.as<float2>();
    p.Etab = c.Etab.as<double>();
    p.step = nullptr;
    p.obs = c.obs.as<double>();
    c.red.ensure((size_t)std::max<int64_t>(G, (h.N + 255) / 256) * 3 * sizeof(double));
    p.red = c.red.as<double>();
    p.counter = nullptr;
    p.N = h.N;
    p.Nk = h.Nk;
    p.c1 = h.c1;
    for (int q = 0; q < 4; ++q) p.occ[q] = (float)h.occ[q];
    p.dt = (float)dt;
    p.dirx = (float)dirx;
    p.diry = (float)diry;
    p.stage = 0;
    p.kahan = kahan ? 1 : 0;
    f.part.ensure((size_t)G * std::max<long long>(m.stot, 1) * sizeof(float2));
    f.Xt.ensure((size_t)h.N * sizeof(float2));
    c.sync.ensure(4 * sizeof(unsigned));
    TDAGW_CUDA(cudaMemsetAsync(c.sync.p, 0, 4 * sizeof(unsigned), s));
    a.dSw = c.dS.as<float2>();
    a.part = f.part.as<float2>();
    a.ytil = f.Y.as<float2>();
    a.Xt = f.Xt.as<float2>();
    a.bar_count = reinterpret_cast<unsigned long long*>(c.sync.p);
    a.err = reinterpret_cast<int*>(c.sync.as<unsigned>() + 2);
    a.T = T;
    a.nslots = nslots;
    a.slot_bytes = slot_bytes;
    a.kmax = kmax;
    a.zs_len = zs_len;
    a.upart_len = upart_len;
    // V-pass groups: as many as keep four columns per thread covering the longest V row
    a.vgroups = 1;
    while (a.vgroups < kCW && 4 * (kCons / (2 * a.vgroups)) >= maxv) a.vgroups *= 2;
    a.extra_arrivals = test_timeout ? 1 : 0;
    a.wait_ns = test_timeout ? 20000000ull : 2000000000ull;
    void* args[] = {&a};
    const void* fn = h.Nb == 2 ? (const void*)ch_persistent_kernel<2> : (const void*)ch_persistent_kernel<4>;
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThr, smem));
    if (per_sm < 1) return false;
    TDAGW_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kThr), args, smem, s));
    c.persistent_launched = true;
    return true;
}

}  // namespace tdagw
