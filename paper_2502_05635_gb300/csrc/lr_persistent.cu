// Persistent low-rank TD-aGW propagation (single trajectory, complex64): one cooperative
// launch runs all RK4 steps of a call.  Per stage (Eq. svd_acc applied to Eq. sigma-from-k,
// inside the RK4 update of Eq. tdagw):
//
//   V pass   y_c = sum_{i in rows(c)} conj(V_i) x_i          (each CTA: its rows)
//   grid barrier; y = sum_c y_c, scaled by S (each CTA: a slice of columns)
//   grid barrier; U pass  dSigma_i = U_i . (S o y) + K^diag_i x_i  (same rows)
//   commutator, RK4 stage update, observables for the same rows
//
// Each CTA owns the pair elements of a contiguous range of k-points, so its commutators use
// only rows it computed and the next stage's V pass needs only its own rows: two grid
// barriers per stage.  The factors U and V (N x ldu complex64, row-major) are the only
// large operands; a CTA's operand stream is two contiguous byte ranges per stage.  A
// producer warp streams them through a shared-memory ring with 1D TMA bulk copies (cp.async.bulk) completing on mbarriers; sixteen consumer warps compute
// from shared memory.  The producer never depends on data, so it keeps copies in flight
// across the grid barriers and HBM stays busy while the barriers resolve.
//
// Every wait is bounded (a budget in ns of %globaltimer): on expiry the CTA records an
// error word, raises its abort flag, stops issuing copies, waits for the copies it has in
// flight and returns; the host reports TDAGW_ERR_TIMEOUT.
#include <algorithm>

#include "common.cuh"
#include "persist.cuh"
#include "stage.cuh"

namespace tdagw {

namespace {

using namespace persist;

constexpr int kConsumerWarps = 16;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;
constexpr int kSlotTarget = 32768;  // bytes per ring slot (whole rows)

// Optional phase timestamps (build with -DTDAGW_TRACE): thread 0 of every CTA records
// %globaltimer at ten points of each of the first kTraceStages stages.
#ifdef TDAGW_TRACE
constexpr int kTraceStages = 16;
__device__ unsigned long long g_trace[160 * kTraceStages * 10];
#define TDAGW_TRACE_POINT(k)                                                                \
    do {                                                                                    \
        if (tid == 0 && cta < 160 && n * 4 + st < kTraceStages)                             \
            g_trace[(cta * kTraceStages + n * 4 + st) * 10 + (k)] = gtimer();               \
    } while (0)
#else
#define TDAGW_TRACE_POINT(k) \
    do {                     \
    } while (0)
#endif

struct LRArgs {
    const float2* U;
    const float2* V;
    const float* S;
    const float2* diag;
    const float2* kblk;  // k-block reading of K^diag (Nk x P x P), or nullptr: diag
    StageParams<float> sp;
    float2* dSw;         // dSigma written by the U pass (sp.dS reads it)
    float2* part;        // gridDim x ldu partial y vectors
    float2* ytil;        // ldu, S o y
    unsigned long long* bar_count;  // monotonic arrival counter of the grid barrier
    int* err;
    int64_t N;
    int Nk, r, ldu, T;
    int rows_per_slot, nslots, slot_bytes, rows_max;
    int u_parts, u_part_w;  // U pass: column parts per row (power of 2) and their width
    int extra_arrivals;  // > 0 only for the timeout test: the barrier can never complete
    unsigned long long wait_ns;
};

#ifndef TDAGW_LR_EVICT_FIRST
#define TDAGW_LR_EVICT_FIRST 1  // factor rows streamed with an L2 evict-first policy (read once per stage)
#endif
__device__ __forceinline__ void consumer_sync() { named_sync<kConsumers>(); }

// Grid-wide barrier among the consumer threads of all CTAs (monotonic arrival counter; see
// persist::grid_sync).  Returns false (and raises abort) if it did not complete in time.
__device__ __forceinline__ bool grid_sync(const LRArgs& a, unsigned& lgen, volatile int* abort_s) {
    return persist::grid_sync<kConsumers>(a.bar_count, a.err, a.extra_arrivals, a.wait_ns, lgen, abort_s);
}

// Observables row `row` from the per-CTA partials (one warp; fixed summation order).
__device__ __forceinline__ void reduce_step_obs(const LRArgs& a, int G, int lane, int row) {
    reduce_obs_row(a.sp.red, G, 1.0 / (double)a.Nk, a.sp.obs + 3 * (int64_t)row, lane);
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 1) lr_persistent_kernel(LRArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    // rows of this CTA: all pair elements of the k-points [ka, kb), so the commutator of
    // every k it owns needs only rows it computed itself (no grid barrier between the
    // U pass and the next V pass)
    const int64_t ka = (int64_t)cta * a.Nk / G, kb = (int64_t)(cta + 1) * a.Nk / G;
    const int64_t ra = ka * NB * NB, rb = kb * NB * NB;
    const int nrows = (int)(rb - ra);
    const int rps = a.rows_per_slot, ns = a.nslots, ldu = a.ldu;
    const int ntiles = (nrows + rps - 1) / rps;

    unsigned char* ring = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)ns * a.slot_bytes);
    uint64_t* empty = full + ns;
    // partial U-pass dot products: rows_max x u_parts (at least ldu entries of room)
    float2* upart = reinterpret_cast<float2*>(empty + ns);
    float2* xs = upart + max(ldu, a.rows_max * a.u_parts);
    double* wred = reinterpret_cast<double*>(xs + a.rows_max);
    volatile int* abort_s = reinterpret_cast<volatile int*>(wred + 3 * kConsumerWarps);

    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kConsumerWarps);
        }
        *abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ------------------------------------------------------------ producer warp
        if (lane == 0) {
            RingPos pos{0, 0u};
            uint64_t issued = 0;
            bool ok = true;
            uint64_t policy = 0;
            if (TDAGW_LR_EVICT_FIRST) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));

            for (int n = 0; n < a.T && ok; ++n)
                for (int st = 0; st < 4 && ok; ++st)
                    for (int pass = 0; pass < 2 && ok; ++pass) {
                        const float2* base = (pass == 0 ? a.V : a.U) + ra * ldu;
                        for (int t = 0; t < ntiles; ++t) {
                            if (issued >= (uint64_t)ns &&
                                !mbar_wait(empty + pos.slot, pos.phase ^ 1u, abort_s, a.wait_ns)) {
                                ok = false;
                                break;
                            }
                            const int r0 = t * rps;
                            const int nr = min(rps, nrows - r0);
                            const uint32_t bytes = (uint32_t)nr * ldu * 8u;
                            mbar_expect_tx(full + pos.slot, bytes);
                            if (TDAGW_LR_EVICT_FIRST)
                                bulk_g2s_hint(ring + (size_t)pos.slot * a.slot_bytes, base + (int64_t)r0 * ldu,
                                              bytes, full + pos.slot, policy);
                            else
                                bulk_g2s(ring + (size_t)pos.slot * a.slot_bytes, base + (int64_t)r0 * ldu,
                                         bytes, full + pos.slot);
                            ++issued;
                            pos.advance(1, ns);
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
        const int64_t ea = ra, eb = rb;
        const int jr0 = (int)((int64_t)cta * a.r / G), jr1 = (int)((int64_t)(cta + 1) * a.r / G);
        unsigned lgen = 0;
        RingPos pos{0, 0u};
        bool ok = true;
        for (int e = tid; e < nrows; e += kConsumers) xs[e] = __ldcg(a.sp.X + ra + e);
        consumer_sync();
        for (int n = 0; n < a.T && ok; ++n) {
            for (int st = 0; st < 4 && ok; ++st) {
                TDAGW_TRACE_POINT(0);
                // ---- V pass: every warp reads every row; thread owns column pairs
                //      tid and tid + 512 (ldu <= 2048)
                float2 acc[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
                for (int t = 0; t < ntiles; ++t) {
                    if (!warp_wait_full(full, pos, abort_s, a.wait_ns, lane)) break;
                    const float2* tile = reinterpret_cast<const float2*>(ring + (size_t)pos.slot * a.slot_bytes);
                    const int r0 = t * rps, nr = min(rps, nrows - r0);
                    for (int rr = 0; rr < nr; ++rr) {
                        const float2 xi = xs[r0 + rr];
                        const float2* row = tile + (size_t)rr * ldu;
#pragma unroll
                        for (int m = 0; m < 2; ++m) {
                            const int p = tid + m * kConsumers;
                            if (2 * p < ldu) {
                                const float4 v = *reinterpret_cast<const float4*>(row + 2 * p);
                                acc[2 * m] = cfmac(make_float2(v.x, v.y), xi, acc[2 * m]);
                                acc[2 * m + 1] = cfmac(make_float2(v.z, v.w), xi, acc[2 * m + 1]);
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty + pos.slot);
                    pos.advance(1, ns);
                }
                TDAGW_TRACE_POINT(1);
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int p = tid + m * kConsumers;
                    if (2 * p < ldu)
                        *reinterpret_cast<float4*>(a.part + (size_t)cta * ldu + 2 * p) =
                            make_float4(acc[2 * m].x, acc[2 * m].y, acc[2 * m + 1].x, acc[2 * m + 1].y);
                }
                if (!(ok = grid_sync(a, lgen, abort_s))) break;
                TDAGW_TRACE_POINT(2);
                // observables of the previous step (all CTAs published their partials at its
                // last stage, before this barrier); the last warp is idle in the y sum below
                if (st == 0 && n > 0 && cta == 0 && warp == kConsumerWarps - 1)
                    reduce_step_obs(a, G, lane, n);
                // ---- y = S o sum_c y_c for this CTA's columns, fixed summation order
                for (int j = jr0 + warp; j < jr1; j += kConsumerWarps) {
                    float2 s = make_float2(0.f, 0.f);
                    for (int c2 = lane; c2 < G; c2 += 32) s = cadd(s, __ldcg(a.part + (size_t)c2 * ldu + j));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s = cadd(s, shfl_xor(s, o));
                    if (lane == 0) a.ytil[j] = cscale(s, a.S[j]);
                }
                if (!(ok = grid_sync(a, lgen, abort_s))) break;
                TDAGW_TRACE_POINT(3);
                // ---- U pass: the rows of a tile are split over all consumer warps by
                //      column parts (warp = (row in tile) x parts + part), so a tile is
                //      released as soon as the 16 short partial dot products are done;
                //      each warp keeps its slice of S o y in registers.  Every warp still
                //      observes every tile's phase in order (an mbarrier parity wait is
                //      only unambiguous for a waiter that saw the slot's previous use).
                const int cp = a.u_parts, pw = a.u_part_w;
                const int myq = warp % cp, myr = warp / cp, rstride = kConsumerWarps / cp;
                const int c0 = myq * pw, c1 = min(ldu, c0 + pw);
                float4 yv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int col = c0 + 2 * (lane + 32 * k);
                    yv[k] = col < c1 ? __ldcg(reinterpret_cast<const float4*>(a.ytil + col))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                TDAGW_TRACE_POINT(4);
                for (int t = 0; t < ntiles; ++t) {
                    if (!warp_wait_full(full, pos, abort_s, a.wait_ns, lane)) break;
                    const float2* tile = reinterpret_cast<const float2*>(ring + (size_t)pos.slot * a.slot_bytes);
                    const int r0 = t * rps, nr = min(rps, nrows - r0);
                    for (int rr = myr; rr < nr; rr += rstride) {
                        const float2* ur = tile + (size_t)rr * ldu;
                        float2 d = make_float2(0.f, 0.f), d1 = d;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int col = c0 + 2 * (lane + 32 * k);
                            if (col < c1) {
                                const float4 u = *reinterpret_cast<const float4*>(ur + col);
                                d = cfma(make_float2(u.x, u.y), make_float2(yv[k].x, yv[k].y), d);
                                d1 = cfma(make_float2(u.z, u.w), make_float2(yv[k].z, yv[k].w), d1);
                            }
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
                TDAGW_TRACE_POINT(5);
                consumer_sync();  // all partial dot products of this CTA's rows are in
                // dSigma = sum of the parts (fixed order) + K^diag x (the strict diagonal, or
                // the k = k' block of the row's k-point)
                for (int row = tid; row < nrows; row += kConsumers) {
                    float2 sum = upart[row * cp];
                    for (int q = 1; q < cp; ++q) sum = cadd(sum, upart[row * cp + q]);
                    const int64_t i = ra + row;
                    if (a.kblk) {
                        constexpr int P = NB * NB;
                        const int kk = row / P;
                        const float2* bk = a.kblk + (ra + row) * P;
#pragma unroll
                        for (int q = 0; q < P; ++q) sum = cfma(bk[q], xs[kk * P + q], sum);
                        a.dSw[i] = sum;
                    } else {
                        a.dSw[i] = cfma(a.diag[i], xs[row], sum);
                    }
                }
                consumer_sync();  // this CTA's dSigma rows are complete
                TDAGW_TRACE_POINT(6);
                // ---- commutator + RK4 stage update for k in [ka, kb)
                const int eoff = st == 0 ? 0 : (st == 3 ? 2 : 1);
                const float E = (float)a.sp.Etab[2 * (int64_t)n + eoff];
                ObsDF ob;  // double-float sums (FP64 is slow on this GPU)
                for (int64_t b = ea; b < eb; b += kConsumers) {
                    const int64_t i = b + tid;
                    stage_element<float, NB>(a.sp, i, i < eb, lane, st, E, ob);
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
                    consumer_sync();
                    if (tid == 0) {
                        ObsDF s;
                        for (int w = 0; w < kConsumerWarps; ++w) {
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
                TDAGW_TRACE_POINT(7);
                consumer_sync();
                TDAGW_TRACE_POINT(8);
                for (int e = tid; e < nrows; e += kConsumers) xs[e] = __ldcg(a.sp.X + ra + e);
                consumer_sync();
                TDAGW_TRACE_POINT(9);
            }
        }
        // observables of the last step: every CTA's partial is published by one more barrier
        if (ok && a.T > 0) {
            ok = grid_sync(a, lgen, abort_s);
            if (ok && cta == 0 && warp == 0) reduce_step_obs(a, G, lane, a.T);
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
extern "C" int tdagw_debug_trace(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_trace, sizeof(unsigned long long) * (size_t)n) == cudaSuccess ? 0 : -3;
}
#endif

// Host side: launch geometry, shared-memory ring sizing, cooperative launch.  Returns false
// when the path does not apply (rank too large, too little shared memory), in which case
// the caller uses the stage-wise kernels.
bool launch_lr_persistent(Ctx& c, int T, double dt, double dirx, double diry, bool kahan,
                          bool test_timeout, cudaStream_t s) {
    const HostModel& h = c.hm;
    const int r = c.rank, ldu = r + (r & 1);
    if (c.dtype != TDAGW_C64 || ldu > 2048 || r < 1) return false;
    int dev = 0, nsm = 0, smem_max = 0, coop = 0;
    TDAGW_CUDA(cudaGetDevice(&dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return false;
    const int G = (int)std::min<int64_t>(nsm, h.Nk);          // every CTA owns >= 1 k-point
    const int rows_max = (int)((h.Nk + G - 1) / G) * h.Nb * h.Nb;
    const int row_bytes = ldu * 8;
    int rps = 1;  // rows per slot
    while (rps < 64 && 2 * rps * row_bytes <= kSlotTarget) rps *= 2;
    const int slot_bytes = rps * row_bytes;
    // U pass: rows per slot x column parts = 16 consumer warps (parts of even width)
    const int u_parts = rps >= kConsumerWarps ? 1 : kConsumerWarps / rps;
    const int u_part_w = ((ldu + u_parts - 1) / u_parts + 1) / 2 * 2;
    const size_t extras = (size_t)std::max(ldu, rows_max * u_parts) * 8 + (size_t)rows_max * 8 +
                          3 * kConsumerWarps * 8 + 16;
    const size_t avail = (size_t)smem_max - 1024;
    if (avail < extras + 4 * (size_t)slot_bytes) return false;
    const int nslots = (int)std::min<size_t>(64, (avail - extras) / (slot_bytes + 16));
    const size_t smem = (size_t)nslots * slot_bytes + 16 * (size_t)nslots + extras;

    LRArgs a{};
    a.U = c.U.as<float2>();
    a.dSw = c.dS.as<float2>();
    a.V = c.V.as<float2>();
    a.S = c.S.as<float>();
    a.diag = c.diagF.as<float2>();
    a.kblk = c.kdiag ? c.kblkF.as<float2>() : nullptr;
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
    c.pbuf.ensure((size_t)G * ldu * sizeof(float2));
    c.sync.ensure(4 * sizeof(unsigned));
    TDAGW_CUDA(cudaMemsetAsync(c.sync.p, 0, 4 * sizeof(unsigned), s));
    a.part = c.pbuf.as<float2>();
    a.ytil = c.ytil.as<float2>();
    a.bar_count = reinterpret_cast<unsigned long long*>(c.sync.p);
    a.err = reinterpret_cast<int*>(c.sync.as<unsigned>() + 2);
    a.N = h.N;
    a.Nk = h.Nk;
    a.r = r;
    a.ldu = ldu;
    a.T = T;
    a.rows_per_slot = rps;
    a.nslots = nslots;
    a.slot_bytes = slot_bytes;
    a.rows_max = rows_max;
    a.u_parts = u_parts;
    a.u_part_w = u_part_w;
    a.extra_arrivals = test_timeout ? 1 : 0;
    a.wait_ns = test_timeout ? 20000000ull : 2000000000ull;
    void* args[] = {&a};
    const void* fn = h.Nb == 2 ? (const void*)lr_persistent_kernel<2> : (const void*)lr_persistent_kernel<4>;
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
    if (per_sm < 1) return false;
    TDAGW_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kThreads), args, smem, s));
    c.persistent_launched = true;
    return true;
}

}  // namespace tdagw
