// Batched TD-aGW propagation: B trajectories (different pulses and lengths) in one
// persistent cooperative launch (complex64).  Across trajectories the contraction of Eq.
// sigma-from-k becomes a matrix product: with the states as columns of X (N x B),
//   low rank (Eq. svd_acc):  Y = S o (V^H X)  (r x B),   dSigma = K^diag o X + U Y
//   dense:                   dSigma = K X
// followed by the per-k commutator and RK4 stage update of Eq. tdagw for every column.
//
// Work split: CTA (rg, tg) owns the pair elements of a k-aligned row group rg and the
// trajectories of group tg; trajectories are sorted by length (longest first), so the
// active ones at step n are a prefix of length B_act(n) and each group takes an equal
// share of that prefix -- finished trajectories cost nothing (compaction by sorting).
// Per low-rank stage:
//   A  P[rg] = V[rows(rg)]^H X[rows(rg), tg]        (partial over the row group)
//   -- grid barrier --
//   C  Y[j, tg] = S_j sum_rg P[rg][j, tg]            (each CTA: a slice of j)
//   -- grid barrier --
//   D  dSigma[rows(rg), tg] = U[rows(rg)] Y[:, tg] + K^diag o X
//   E  commutator + RK4 for k in rg, trajectories in tg (rows this CTA just computed)
// Dense stages: grid barrier (X complete), dSigma[rows(rg), tg] = K[rows(rg)] X[:, tg], E.
// The matrix products are register-tiled (4 x 4 complex outputs per thread) FP32 FMAs
// through shared memory.  Grid barriers are bounded waits (as in the single-trajectory
// persistent kernel); on expiry the kernel sets an error word and returns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batched_common.cuh"

namespace tdagw {

using namespace batched;

namespace {

// Commutator + RK4 stage update of one (k, trajectory) block, all NB^2 elements in
// registers (the same arithmetic as stage_element, Eq. tdagw).  The observables (last
// stage) are added to ob in double-float (FP64 arithmetic is slow on this GPU).
template <int NB>
__device__ void stage_kb(const BatchArgs& a, int k, int b, int st, float E, float2 dr, ObsDF& ob) {
    constexpr int NB2 = NB * NB;
    const int64_t Bp = a.Bp;
    float2 X[NB2], M[NB2];
#pragma unroll
    for (int g = 0; g < NB2; ++g) {
        const int64_t i = (int64_t)k * NB2 + g;
        X[g] = __ldcg(a.X + i * Bp + b);
        const float2 d1 = a.dx[i], d2 = a.dy[i];
        const float2 ds = __ldcg(a.dS + i * Bp + b);
        M[g] = make_float2(ds.x + E * (dr.x * d1.x + dr.y * d2.x), ds.y + E * (dr.x * d1.y + dr.y * d2.y));
    }
#pragma unroll
    for (int n = 0; n < NB; ++n)
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            const int g = n * NB + m;
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
            const float2 xs = __ldcg(a.Ssum + e), xc = __ldcg(a.Ccomp + e);
            float2 Xn;
            if (st < 3) {
                const float2 ac = st == 0 ? kv : cadd(__ldcg(a.acc + e), cscale(kv, 2.f));
                a.acc[e] = ac;
                const float cn = st == 2 ? a.dt : 0.5f * a.dt;
                Xn = cadd(xs, cadd(xc, cscale(kv, cn)));
            } else {
                const float2 ac = cadd(__ldcg(a.acc + e), kv);
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
        }
}

// CH: the channel-wise mode (a separate instantiation, so the other modes' code is unchanged)
template <int NB, bool CH>
__global__ void __launch_bounds__(kBThreads, 1) batched_kernel(BatchArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    float2* sA = sm;                       // kChunk x kLdA
    float2* sB = sA + kChunk * kLdA;       // kChunk x 32
    double* sred = reinterpret_cast<double*>(sA + kGemmSmem);  // 16 x kTileB x 3
    __shared__ int abort_s;
    const int tid = threadIdx.x;
    const int rg = blockIdx.x % a.Rg, tg = blockIdx.x / a.Rg;
    const int ka = (int)((int64_t)rg * a.Nk / a.Rg), kb = (int)((int64_t)(rg + 1) * a.Nk / a.Rg);
    const int NB2 = NB * NB;
    const int64_t ra = (int64_t)ka * NB2;
    const int nrows = (kb - ka) * NB2;
    const int jr0 = (int)((int64_t)rg * a.r / a.Rg), jr1 = (int)((int64_t)(rg + 1) * a.r / a.Rg);
    if (tid == 0) abort_s = 0;
    __syncthreads();
    unsigned gen = 0;
    bool ok = true;
    int prev_act = -1;
    for (int n = 0; n < a.Tmax && ok; ++n) {
        const int Bact = a.act[a.n0 + n];
        int b0, b1;
        group_range(Bact, a.Tg, tg, b0, b1);
        const int nb = b1 - b0;
        if (a.ckS && (a.n0 + n) % a.ck_period == 0) {
            // checkpoint of the compensated state at the start of step n0 + n (own block)
            const int64_t slot = (int64_t)((a.n0 + n) / a.ck_period) * a.N * a.Bp;
            for (int e = threadIdx.x; e < nrows * nb; e += kBThreads) {
                const int64_t off = (ra + e / nb) * a.Bp + b0 + e % nb;
                a.ckS[slot + off] = __ldcg(a.Ssum + off);
                a.ckC[slot + off] = __ldcg(a.Ccomp + off);
            }
        }
        for (int st = 0; st < 4 && ok; ++st) {
            // the dense product and the channel-wise row shares read every CTA's rows of X
            const bool need_x_barrier = (a.mode == TDAGW_FULL || CH) ? !(n == 0 && st == 0)
                                                                     : (st == 0 && Bact != prev_act && n > 0);
            if (need_x_barrier && !(ok = bgrid_sync(a, gen, &abort_s))) break;
            if (st == 0 && n > 0 && rg == 0 && a.mode == TDAGW_FULL) {
                // observables of step n-1 for this group's trajectories at that step
                int p0, p1;
                group_range(a.act[a.n0 + n - 1], a.Tg, tg, p0, p1);
                for (int b = p0 + tid; b < p1; b += kBThreads) {
                    double s0 = 0, s1 = 0, s2 = 0;
                    for (int g2 = 0; g2 < a.Rg; ++g2) {
                        s0 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3);
                        s1 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3 + 1);
                        s2 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3 + 2);
                    }
                    double* o = a.obs + ((int64_t)n * a.B + b) * 3;
                    o[0] = s0 / a.Nk;
                    o[1] = s1 / a.Nk;
                    o[2] = s2 / a.Nk;
                }
            }
            if (a.mode != TDAGW_FULL) {
                // A: partial V^H X over this row group (channel-wise: one product per input
                // pair q, its V segment's rows of this row group with the rows k P + q of X)
                if constexpr (!CH) {
                    if (nb > 0)
                        block_gemm<true>(a.V + ra * a.ldu, a.ldu, a.r, nrows, a.X + ra * a.Bp + b0, a.Bp, nb,
                                         a.P + (int64_t)rg * a.r * a.Bp + b0, a.Bp, false, nullptr, nullptr,
                                         sA, sB);
                } else if (nb > 0) {
                    // channel-wise: q-major row shares as in D below (rows q Nk + k' of the
                    // V segments, one or two input pairs per row group); the group writes the
                    // partials of those pairs' columns only
                    const int u0 = (int)((int64_t)rg * a.N / a.Rg), u1 = (int)((int64_t)(rg + 1) * a.N / a.Rg);
                    for (int q = u0 / a.Nk; q < NB2 && q * a.Nk < u1; ++q) {
                        const int ldv = a.chm->ldv[q];
                        const int k0 = max(u0 - q * a.Nk, 0), k1 = min(u1 - q * a.Nk, a.Nk);
                        if (ldv == 0 || k1 <= k0) continue;
                        block_gemm<true>(a.Vch + a.chm->vbase[q] + (int64_t)k0 * ldv, ldv, ldv, k1 - k0,
                                         a.X + ((int64_t)k0 * NB2 + q) * a.Bp + b0, (int64_t)NB2 * a.Bp, nb,
                                         a.P + ((int64_t)rg * a.r + a.chm->sbase[q]) * a.Bp + b0, a.Bp, false,
                                         nullptr, nullptr, sA, sB);
                    }
                }
                if (!(ok = bgrid_sync(a, gen, &abort_s))) break;
                if (st == 0 && n > 0 && rg == 0) {
                    int p0, p1;
                    group_range(a.act[a.n0 + n - 1], a.Tg, tg, p0, p1);
                    for (int b = p0 + tid; b < p1; b += kBThreads) {
                        double s0 = 0, s1 = 0, s2 = 0;
                        for (int g2 = 0; g2 < a.Rg; ++g2) {
                            s0 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3);
                            s1 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3 + 1);
                            s2 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3 + 2);
                        }
                        double* o = a.obs + ((int64_t)n * a.B + b) * 3;
                        o[0] = s0 / a.Nk;
                        o[1] = s1 / a.Nk;
                        o[2] = s2 / a.Nk;
                    }
                }
                // C: Y[j][b] = S_j sum over row groups, j in this CTA's slice (channel-wise:
                // over the row groups whose share touches the input pair of column j)
                for (int e = tid; e < (jr1 - jr0) * nb; e += kBThreads) {
                    const int j = jr0 + e / nb, b = b0 + e % nb;
                    int g0 = 0, g1 = a.Rg - 1;
                    if constexpr (CH) {
                        int q = 0;
                        while (q + 1 < NB2 && a.chm->sbase[q + 1] <= j) ++q;
                        const int64_t NR = a.N, RG = a.Rg, lo = (int64_t)q * a.Nk;
                        g0 = max(0, (int)(((lo + 1) * RG + NR - 1) / NR) - 1);
                        g1 = min(a.Rg - 1, (int)(((lo + a.Nk) * RG + NR - 1) / NR) - 1);
                    }
                    float2 s = make_float2(0.f, 0.f);
                    for (int g2 = g0; g2 <= g1; ++g2)
                        s = cadd(s, __ldcg(a.P + ((int64_t)g2 * a.r + j) * a.Bp + b));
                    a.Y[(int64_t)j * a.Bp + b] = cscale(s, a.S[j]);
                }
                if (!(ok = bgrid_sync(a, gen, &abort_s))) break;
                if constexpr (!CH) {
                    // D: dSigma = U Y + K^diag X for this row group (the strict diagonal fused
                    // into the product, or the k = k' blocks added after it)
                    if (nb > 0)
                        block_gemm<false>(a.U + ra * a.ldu, a.ldu, nrows, a.r, a.Y + b0, a.Bp, nb,
                                          a.dS + ra * a.Bp + b0, a.Bp, a.kblk == nullptr, a.diag + ra,
                                          a.X + ra * a.Bp + b0, sA, sB);
                    if (a.kblk) {
                        __syncthreads();  // this CTA's U Y rows are written
                        if (nb > 0) kblock_term<NB, false>(a.kblk, a.X, a.dS, a.Bp, ra, nrows, b0, nb);
                    }
                } else {
                    // D (channel-wise) by p-major shares: row group rg takes the rows
                    // [u0, u1) of the order p Nk + k (one or two output pairs), so each pair
                    // is one product over many k-points instead of the group's few: the dense
                    // diagonal channel with x_p over all k, then each off-diagonal channel's
                    // U^pq with its block of S o Y added.  The rows reach their k-point's
                    // owner through global memory across the barrier below.
                    const int64_t ldo = (int64_t)NB2 * a.Bp;
                    const int u0 = (int)((int64_t)rg * a.N / a.Rg), u1 = (int)((int64_t)(rg + 1) * a.N / a.Rg);
                    if (nb > 0)
                        for (int p = u0 / a.Nk; p < NB2 && p * a.Nk < u1; ++p) {
                            const int k0 = max(u0 - p * a.Nk, 0), k1 = min(u1 - p * a.Nk, a.Nk);
                            if (k1 <= k0) continue;
                            const int ldw = a.chm->ldw[p], nl = a.chm->nlr[p];
                            const float2* Ub = a.Uch + a.chm->ubase[p] + (int64_t)k0 * ldw;
                            float2* o = a.dS + ((int64_t)k0 * NB2 + p) * a.Bp + b0;
                            block_gemm<false>(Ub + nl, ldw, k1 - k0, a.Nk, a.X + (int64_t)p * a.Bp + b0, ldo, nb, o,
                                              ldo, false, nullptr, nullptr, sA, sB);
                            for (int q = 0; q < NB2; ++q) {
                                const int z = a.choff[2 * NB2 * NB2 + p * NB2 + q];
                                if (q == p || z == 0) continue;
                                const int64_t yrow = a.chm->sbase[q] + a.choff[NB2 * NB2 + q * NB2 + p];
                                block_gemm<false, true>(Ub + a.choff[p * NB2 + q], ldw, k1 - k0, z,
                                                        a.Y + yrow * a.Bp + b0, a.Bp, nb, o, ldo, false, nullptr,
                                                        nullptr, sA, sB);
                            }
                        }
                    // every CTA has read all rows of X before any CTA rewrites its rows
                    if (!(ok = bgrid_sync(a, gen, &abort_s))) break;
                }
            } else {
                if (nb > 0)
                    block_gemm<false>(a.K + ra * a.N, a.N, nrows, (int)a.N, a.X + b0, a.Bp, nb,
                                      a.dS + ra * a.Bp + b0, a.Bp, false, nullptr, nullptr, sA, sB);
                // every CTA has read all rows of X before any CTA rewrites its rows
                if (!(ok = bgrid_sync(a, gen, &abort_s))) break;
            }
            __syncthreads();
            if (a.recX) {
                // stage input and dSigma of this stage, for the adjoint's backward sweep
                const int64_t slot = (int64_t)(n * 4 + st) * a.N * a.Bp;
                for (int e = threadIdx.x; e < nrows * nb; e += kBThreads) {
                    const int64_t off = (ra + e / nb) * a.Bp + b0 + e % nb;
                    a.recX[slot + off] = __ldcg(a.X + off);
                    a.recDS[slot + off] = __ldcg(a.dS + off);
                }
            }
            // E: commutator + RK4 for (k in [ka, kb), b in [b0, b1))
            const int eoff = st == 0 ? 0 : (st == 3 ? 2 : 1);
            {
                const int bl = tid % kTileB, kg = tid / kTileB;  // 16 k-groups x 32 trajectories
                ObsDF ob;
                if (bl < nb) {
                    const int b = b0 + bl;
                    const float E = (float)a.Etab[(int64_t)b * a.ldE + 2 * (a.n0 + n) + eoff];
                    const float2 dr = a.dir[b];
                    for (int k = ka + kg; k < kb; k += kBThreads / kTileB) stage_kb<NB>(a, k, b, st, E, dr, ob);
                }
                if (st == 3) {
                    sred[(kg * kTileB + bl) * 3] = ob.p.value();
                    sred[(kg * kTileB + bl) * 3 + 1] = ob.j.value();
                    sred[(kg * kTileB + bl) * 3 + 2] = ob.o.value();
                }
            }
            __syncthreads();
            if (st == 3)
                for (int bl = tid; bl < nb; bl += kBThreads) {
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                    for (int kg = 0; kg < kBThreads / kTileB; ++kg) {
                        s0 += sred[(kg * kTileB + bl) * 3];
                        s1 += sred[(kg * kTileB + bl) * 3 + 1];
                        s2 += sred[(kg * kTileB + bl) * 3 + 2];
                    }
                    double* rr = a.red + ((int64_t)rg * a.Bp + b0 + bl) * 3;
                    rr[0] = s0;
                    rr[1] = s1;
                    rr[2] = s2;
                }
            __syncthreads();
        }
        prev_act = Bact;
    }
    // observables of the last step
    if (ok && a.Tmax > 0 && bgrid_sync(a, gen, &abort_s) && rg == 0) {
        const int n = a.Tmax;
        int p0, p1;
        group_range(a.act[a.n0 + n - 1], a.Tg, tg, p0, p1);
        for (int b = p0 + tid; b < p1; b += kBThreads) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int g2 = 0; g2 < a.Rg; ++g2) {
                s0 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3);
                s1 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3 + 1);
                s2 += __ldcg(a.red + ((int64_t)g2 * a.Bp + b) * 3 + 2);
            }
            double* o = a.obs + ((int64_t)n * a.B + b) * 3;
            o[0] = s0 / a.Nk;
            o[1] = s1 / a.Nk;
            o[2] = s2 / a.Nk;
        }
    }
}

}  // namespace

}  // namespace tdagw

namespace tdagw {

namespace {

__global__ void replicate_rows_kernel(const double* __restrict__ row, double* __restrict__ obs, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        obs[3 * b] = row[0];
        obs[3 * b + 1] = row[1];
        obs[3 * b + 2] = row[2];
    }
}

// obs_out[n][perm[b]] = obs_sorted[n][b]
__global__ void unpermute_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                 const int* __restrict__ perm, int B, int64_t rows) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * B) return;
    const int64_t n = e / B;
    const int b = (int)(e % B);
    for (int q = 0; q < 3; ++q) dst[(n * B + perm[b]) * 3 + q] = src[e * 3 + q];
}

struct BatchPlan {
    int Rg = 0, Tg = 0;
};

}  // namespace

// Host driver of the batched path (complex64 contexts).  Trajectories are sorted by length
// (longest first); the block shape (row groups x trajectory groups) is picked by timing a
// few steps of each candidate (cached per context for this mode, batch size and rank).
BatchSetup prepare_batch(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt) {
    const HostModel& h = c.hm;
    cudaStream_t s = c.stream;
    const int64_t N = h.N;
    BatchSetup bs;
    std::vector<int>& perm = bs.perm;
    perm.resize(B);
    for (int b = 0; b < B; ++b) perm[b] = b;
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return steps[x] > steps[y]; });
    const int Tmax = steps[perm[0]];
    const int Bp = (B + 3) / 4 * 4;
    const int64_t ldE = 2 * (int64_t)Tmax + 1;
    std::vector<int>& act = bs.act;
    act.assign(std::max(Tmax, 1), 0);
    for (int n = 0; n < Tmax; ++n) {
        int cnt = 0;
        for (int b = 0; b < B; ++b) cnt += steps[b] > n ? 1 : 0;
        act[n] = cnt;
    }
    // per-trajectory inputs in sorted order
    c.bEtab.ensure((size_t)B * ldE * sizeof(double));
    TDAGW_CUDA(cudaMemsetAsync(c.bEtab.p, 0, (size_t)B * ldE * sizeof(double), s));
    std::vector<float2> dir(B);
    std::vector<FieldParams> fp(B);
    for (int q = 0; q < B; ++q) {
        const tdagw_field& f = fields[perm[q]];
        const int64_t ns = 2 * (int64_t)steps[perm[q]] + 1;
        if (f.kind == TDAGW_FIELD_TABLE)
            TDAGW_CUDA(cudaMemcpyAsync(c.bEtab.as<double>() + (int64_t)q * ldE, f.table, ns * sizeof(double),
                                       cudaMemcpyHostToDevice, s));
        fp[q] = FieldParams{f.E0, f.omega, f.t0, f.sigma, f.T_pulse, f.kind, ns};
        dir[q] = make_float2((float)f.dir_x, (float)f.dir_y);
    }
    // analytic tables of all trajectories in one launch
    c.bfield.ensure(B * sizeof(FieldParams));
    TDAGW_CUDA(cudaMemcpyAsync(c.bfield.p, fp.data(), B * sizeof(FieldParams), cudaMemcpyHostToDevice, s));
    launch_field_tables(c.bfield.as<FieldParams>(), B, ldE, ldE, dt, c.bEtab.as<double>(), s);
    c.bdir.ensure(B * sizeof(float2));
    TDAGW_CUDA(cudaMemcpyAsync(c.bdir.p, dir.data(), B * sizeof(float2), cudaMemcpyHostToDevice, s));
    c.bact.ensure(act.size() * sizeof(int));
    TDAGW_CUDA(cudaMemcpyAsync(c.bact.p, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    c.bperm.ensure(B * sizeof(int));
    TDAGW_CUDA(cudaMemcpyAsync(c.bperm.p, perm.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    // state
    const size_t sbytes = (size_t)N * Bp * sizeof(float2);
    for (DevBuf* b : {&c.bX, &c.bS, &c.bC, &c.bA, &c.bdS}) b->ensure(sbytes);
    // observables: row 0 is the equilibrium value for every trajectory
    const int64_t rows = Tmax + 1;
    c.bobs.ensure((size_t)rows * B * 3 * sizeof(double));
    TDAGW_CUDA(cudaMemsetAsync(c.bobs.p, 0xFF, (size_t)rows * B * 3 * sizeof(double), s));  // NaN
    c.obs.ensure((size_t)std::max<int64_t>(rows * B, 1) * 3 * sizeof(double));
    TDAGW_CUDA(cudaMemsetAsync(c.X.p, 0, N * sizeof(float2), s));
    launch_observables_row<float>(c, c.X.p, 0, s);
    replicate_rows_kernel<<<(B + 127) / 128, 128, 0, s>>>(c.obs.as<double>(), c.bobs.as<double>(), B);
    check_launch("replicate_rows_kernel");
    bs.Tmax = Tmax;
    bs.Bp = Bp;
    bs.ldE = ldE;
    bs.rows = rows;
    return bs;
}

void reset_batch_observables(Ctx& c, const BatchSetup& bs, int B) {
    TDAGW_CUDA(cudaMemsetAsync(c.bobs.p, 0xFF, (size_t)bs.rows * B * 3 * sizeof(double), c.stream));
    replicate_rows_kernel<<<(B + 127) / 128, 128, 0, c.stream>>>(c.obs.as<double>(), c.bobs.as<double>(), B);
    check_launch("replicate_rows_kernel");
}

void launch_batched(Ctx& c, const void* fn, dim3 grid, dim3 block, size_t smem, const void* args,
                    size_t args_size, const std::vector<ResetOp>& resets, bool use_graph) {
    cudaStream_t s = c.stream;
    void* kargs[] = {const_cast<void*>(args)};
    auto direct = [&](cudaStream_t st) {
        for (const ResetOp& r : resets) TDAGW_CUDA(cudaMemsetAsync(r.p, 0, r.bytes, st));
        TDAGW_CUDA(cudaLaunchCooperativeKernel(fn, grid, block, kargs, smem, st));
    };
    if (!use_graph || c.batch_graphs_off) {
        direct(s);
        return;
    }
    // key: kernel, geometry, shared memory, the argument bytes and the reset list
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        key.insert(key.end(), b, b + n);
    };
    put(&fn, sizeof(fn));
    put(&grid, sizeof(grid));
    put(&block, sizeof(block));
    put(&smem, sizeof(smem));
    put(args, args_size);
    for (const ResetOp& r : resets) put(&r, sizeof(r));
    for (size_t i = 0; i < c.batch_graphs.size(); ++i)
        if (c.batch_graphs[i].key == key) {
            TDAGW_CUDA(cudaGraphLaunch(c.batch_graphs[i].exec, s));
            return;
        }
    if (!c.cap) TDAGW_CUDA(cudaStreamCreateWithFlags(&c.cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool ok = cudaStreamBeginCapture(c.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        for (const ResetOp& r : resets) ok = ok && cudaMemsetAsync(r.p, 0, r.bytes, c.cap) == cudaSuccess;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeCooperative;
        attr.val.cooperative = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c.cap;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        ok = ok && cudaLaunchKernelExC(&cfg, fn, kargs) == cudaSuccess;
        const bool ended = cudaStreamEndCapture(c.cap, &g) == cudaSuccess;
        ok = ok && ended && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
    }
    if (!ok) {
        // capture of a cooperative launch unavailable: direct launches from now on
        cudaGetLastError();
        if (ge) cudaGraphExecDestroy(ge);
        c.batch_graphs_off = true;
        direct(s);
        return;
    }
    if (c.batch_graphs.size() >= 8) {
        cudaGraphExecDestroy(c.batch_graphs.front().exec);
        c.batch_graphs.erase(c.batch_graphs.begin());
    }
    c.batch_graphs.push_back({key, ge});
    TDAGW_CUDA(cudaGraphLaunch(ge, s));
}

void finish_batch(Ctx& c, const BatchSetup& bs, int B) {
    const int64_t rows = bs.rows;
    c.obs.ensure((size_t)rows * B * 3 * sizeof(double));
    unpermute_kernel<<<(unsigned)((rows * B + 255) / 256), 256, 0, c.stream>>>(
        c.bobs.as<double>(), c.obs.as<double>(), c.bperm.as<int>(), B, rows);
    check_launch("unpermute_kernel");
    c.obs_rows = rows;
    c.obs_B = B;
}

void propagate_batched(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt,
                       int mode, int flags) {
    TDAGW_REQUIRE(c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED, "batched propagation needs a complex64 context");
    TDAGW_REQUIRE(flags & TDAGW_FLAG_RESET, TDAGW_ERR_UNSUPPORTED,
                  "batched propagation starts from drho = 0 (TDAGW_FLAG_RESET)");
    const HostModel& h = c.hm;
    cudaStream_t s = c.stream;
    const int64_t N = h.N;
    const BatchSetup bs = prepare_batch(c, fields, B, steps, dt);
    const std::vector<int>& perm = bs.perm;
    const int Tmax = bs.Tmax;
    const int Bp = bs.Bp;
    const int64_t ldE = bs.ldE;
    const size_t sbytes = (size_t)N * Bp * sizeof(float2);
    // channel-wise mode: S, the partials and Y span the stot columns of the V segments
    const int r = mode == TDAGW_LOWRANK ? c.rank : (mode == TDAGW_CHANNEL ? (int)c.ch.m.stot : 0);
    const int ldu = r + (r & 1);

    int dev = 0, nsm = 0;
    TDAGW_CUDA(cudaGetDevice(&dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = (size_t)kGemmSmem * sizeof(float2) +
                        (size_t)(kBThreads / kTileB) * kTileB * 3 * sizeof(double);
    const bool ch = mode == TDAGW_CHANNEL;
    const void* fn = h.Nb == 2 ? (ch ? (const void*)batched_kernel<2, true> : (const void*)batched_kernel<2, false>)
                               : (ch ? (const void*)batched_kernel<4, true> : (const void*)batched_kernel<4, false>);
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBThreads, smem));
    TDAGW_REQUIRE(per_sm >= 1, TDAGW_ERR_UNSUPPORTED, "batched kernel does not fit on this device");
    const int max_ctas = nsm * per_sm;

    BatchArgs a{};
    a.U = c.U.as<float2>();
    a.V = c.V.as<float2>();
    a.S = mode == TDAGW_CHANNEL ? c.ch.S.as<float>() : c.S.as<float>();
    a.diag = c.diagF.as<float2>();
    if (mode == TDAGW_CHANNEL) {
        // layout tables on the device: ChMeta, then uoff, voff and z (P x P each)
        const int P = h.Nb * h.Nb;
        std::vector<int> tab(3 * P * P);
        for (int e = 0; e < P * P; ++e) {
            tab[e] = c.ch.uoff[e];
            tab[P * P + e] = c.ch.voff[e];
            tab[2 * P * P + e] = c.ch.z[e];
        }
        c.bchm.ensure(sizeof(ChMeta) + tab.size() * sizeof(int));
        TDAGW_CUDA(cudaMemcpyAsync(c.bchm.p, &c.ch.m, sizeof(ChMeta), cudaMemcpyHostToDevice, s));
        TDAGW_CUDA(cudaMemcpyAsync(static_cast<char*>(c.bchm.p) + sizeof(ChMeta), tab.data(), tab.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, s));
        a.Vch = c.ch.V.as<float2>();
        a.Uch = c.ch.U.as<float2>();
        a.chm = c.bchm.as<ChMeta>();
        a.choff = reinterpret_cast<const int*>(static_cast<char*>(c.bchm.p) + sizeof(ChMeta));
    }
    a.kblk = c.kdiag ? c.kblkF.as<float2>() : nullptr;
    a.K = c.K.as<float2>();
    a.dx = c.dx.as<float2>();
    a.dy = c.dy.as<float2>();
    a.vx = c.vx.as<float2>();
    a.gap = c.gap.as<float2>();
    a.X = c.bX.as<float2>();
    a.Ssum = c.bS.as<float2>();
    a.Ccomp = c.bC.as<float2>();
    a.acc = c.bA.as<float2>();
    a.dS = c.bdS.as<float2>();
    a.Etab = c.bEtab.as<double>();
    a.dir = c.bdir.as<float2>();
    a.act = c.bact.as<int>();
    a.obs = c.bobs.as<double>();
    a.N = N;
    a.ldE = ldE;
    a.Nk = h.Nk;
    a.Nb = h.Nb;
    a.r = r;
    a.ldu = ldu;
    a.Bp = Bp;
    a.B = B;
    a.mode = mode;
    a.kahan = (flags & TDAGW_FLAG_NO_KAHAN) ? 0 : 1;
    a.c1 = h.c1;
    for (int q = 0; q < 4; ++q) a.occ[q] = (float)h.occ[q];
    a.dt = (float)dt;
    a.wait_ns = 2000000000ull;
    c.sync.ensure(4 * sizeof(unsigned));
    a.bar = reinterpret_cast<unsigned long long*>(c.sync.p);
    a.err = reinterpret_cast<int*>(c.sync.as<unsigned>() + 2);

    auto run = [&](const BatchPlan& pl, int T) {
        a.Rg = pl.Rg;
        a.Tg = pl.Tg;
        a.Tmax = T;
        c.bP.ensure((size_t)std::max(1, pl.Rg * std::max(r, 1)) * Bp * sizeof(float2));
        c.bY.ensure((size_t)std::max(r, 1) * Bp * sizeof(float2));
        c.bred.ensure((size_t)pl.Rg * Bp * 3 * sizeof(double));
        a.P = c.bP.as<float2>();
        a.Y = c.bY.as<float2>();
        a.red = c.bred.as<double>();
        launch_batched(c, fn, dim3(pl.Rg * pl.Tg), dim3(kBThreads), smem, &a, sizeof(a),
                       {{c.bX.p, sbytes}, {c.bS.p, sbytes}, {c.bC.p, sbytes}, {c.sync.p, 4 * sizeof(unsigned)}},
                       !(flags & TDAGW_FLAG_NO_GRAPH) && !a.extra_arrivals);
        c.persistent_launched = true;
    };

    const uint64_t key = ((uint64_t)mode << 56) | ((uint64_t)B << 32) | (uint64_t)(uint32_t)r;
    const int tg_min = (B + kTileB - 1) / kTileB;  // at most kTileB trajectories per block
    BatchPlan plan;
    const bool test_timeout = (flags & TDAGW_FLAG_TEST_TIMEOUT) != 0;
    auto it = c.batch_plans.find(key);
    if (test_timeout) {
        // timeout test: the first candidate untuned; the launch below waits for an arrival
        // that never comes
        plan = {std::min(h.Nk, max_ctas / tg_min), tg_min};
    } else if (it != c.batch_plans.end()) {
        plan.Rg = it->second.first;
        plan.Tg = it->second.second;
        TDAGW_REQUIRE(plan.Tg >= tg_min && plan.Rg >= 1 && plan.Rg <= h.Nk && plan.Rg * plan.Tg <= max_ctas,
                      TDAGW_ERR_CUDA, "cached batched launch plan does not fit the call");
    } else {
        // candidates: at most 32 trajectories per block (the register tile), CTAs <= SMs
        std::vector<BatchPlan> cands;
        for (int tg = tg_min; tg <= std::min(B, 8 * tg_min); tg *= 2) {
            const int rg = std::min(h.Nk, max_ctas / tg);
            if (rg >= 1) cands.push_back({rg, tg});
        }
        TDAGW_REQUIRE(!cands.empty(), TDAGW_ERR_UNSUPPORTED, "too many trajectories for one launch");
        if (cands.size() == 1 || Tmax < 8) {
            plan = cands[0];
        } else {
            cudaEvent_t e0, e1;
            TDAGW_CUDA(cudaEventCreate(&e0));
            TDAGW_CUDA(cudaEventCreate(&e1));
            float best = 1e30f;
            for (const BatchPlan& pl : cands) {
                run(pl, 2);  // warm
                TDAGW_CUDA(cudaEventRecord(e0, s));
                run(pl, 6);
                TDAGW_CUDA(cudaEventRecord(e1, s));
                TDAGW_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                TDAGW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    plan = pl;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            int err = 0;
            TDAGW_CUDA(cudaMemcpy(&err, c.sync.as<unsigned>() + 2, sizeof(int), cudaMemcpyDeviceToHost));
            TDAGW_REQUIRE(!err, TDAGW_ERR_TIMEOUT, "a bounded wait gave up while tuning the batched kernel");
            // the tuning runs overwrote the observables: restore the first row
            reset_batch_observables(c, bs, B);
        }
        c.batch_plans[key] = {plan.Rg, plan.Tg};
    }
    const bool ckpt = (flags & TDAGW_FLAG_CHECKPOINT) != 0;
    c.adj.valid = false;
    if (ckpt) {
        // compensated state every ceil(sqrt(Tmax)) steps for the adjoint's recomputes
        const int period = std::max(1, (int)std::ceil(std::sqrt((double)Tmax)));
        const int nck = (Tmax + period - 1) / period;
        c.ckS.ensure((size_t)nck * sbytes);
        c.ckC.ensure((size_t)nck * sbytes);
        a.ckS = c.ckS.as<float2>();
        a.ckC = c.ckC.as<float2>();
        a.ck_period = period;
    }
    if (test_timeout) {
        a.extra_arrivals = 1;
        a.wait_ns = 20000000ull;
    }
    run(plan, Tmax);
    a.extra_arrivals = 0;
    a.wait_ns = 2000000000ull;
    if (ckpt) {
        AdjointState& st = c.adj;
        st.valid = true;
        st.B = B;
        st.Bp = Bp;
        st.Tmax = Tmax;
        st.period = a.ck_period;
        st.Rg = plan.Rg;
        st.Tg = plan.Tg;
        st.mode = mode;
        st.dt = dt;
        st.perm = perm;
        st.steps.assign(steps, steps + B);
        st.fields.assign(fields, fields + B);
        for (tdagw_field& f : st.fields) f.table = nullptr;
        st.fwd_args.resize(sizeof(BatchArgs));
        std::memcpy(st.fwd_args.data(), &a, sizeof(BatchArgs));
        st.fwd_fn = fn;
    }
    c.last_plan_rg = plan.Rg;
    c.last_plan_tg = plan.Tg;
    // observables in the caller's trajectory order
    finish_batch(c, bs, B);
}

}  // namespace tdagw

namespace tdagw {

// The backward sweep of the adjoint after a checkpointed split-FP16 (tensor-core) forward
// run uses the FP32 batched partition: the low-rank plan cached for this batch size and
// rank, else the first candidate shape (at most kTileB trajectories per block, CTAs <=
// SMs).  Fills c.adj like a checkpointed FP32 run; the caller adds the tensor-core fields.
void prepare_adjoint_fp32(Ctx& c, const BatchSetup& bs, const tdagw_field* fields, int B, const int* steps,
                          double dt, int flags) {
    const HostModel& h = c.hm;
    const int64_t N = h.N;
    const int Bp = bs.Bp;
    const int r = c.rank, ldu = r + (r & 1);
    int dev = 0, nsm = 0;
    TDAGW_CUDA(cudaGetDevice(&dev));
    TDAGW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = (size_t)kGemmSmem * sizeof(float2) +
                        (size_t)(kBThreads / kTileB) * kTileB * 3 * sizeof(double);
    const void* fn = h.Nb == 2 ? (const void*)batched_kernel<2, false> : (const void*)batched_kernel<4, false>;
    TDAGW_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TDAGW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBThreads, smem));
    TDAGW_REQUIRE(per_sm >= 1, TDAGW_ERR_UNSUPPORTED, "batched kernel does not fit on this device");
    const int max_ctas = nsm * per_sm;
    const uint64_t key = ((uint64_t)TDAGW_LOWRANK << 56) | ((uint64_t)B << 32) | (uint64_t)(uint32_t)r;
    const int tg_min = (B + kTileB - 1) / kTileB;
    BatchPlan plan;
    auto it = c.batch_plans.find(key);
    if (it != c.batch_plans.end() && it->second.second >= tg_min && it->second.first >= 1 &&
        it->second.first <= h.Nk && it->second.first * it->second.second <= max_ctas) {
        plan.Rg = it->second.first;
        plan.Tg = it->second.second;
    } else {
        plan.Tg = tg_min;
        plan.Rg = std::min(h.Nk, max_ctas / tg_min);
        TDAGW_REQUIRE(plan.Rg >= 1, TDAGW_ERR_UNSUPPORTED, "too many trajectories for one launch");
    }
    BatchArgs a{};
    a.U = c.U.as<float2>();
    a.V = c.V.as<float2>();
    a.S = c.S.as<float>();
    a.diag = c.diagF.as<float2>();
    a.kblk = c.kdiag ? c.kblkF.as<float2>() : nullptr;
    a.K = c.K.as<float2>();
    a.dx = c.dx.as<float2>();
    a.dy = c.dy.as<float2>();
    a.vx = c.vx.as<float2>();
    a.gap = c.gap.as<float2>();
    a.X = c.bX.as<float2>();
    a.Ssum = c.bS.as<float2>();
    a.Ccomp = c.bC.as<float2>();
    a.acc = c.bA.as<float2>();
    a.dS = c.bdS.as<float2>();
    a.Etab = c.bEtab.as<double>();
    a.dir = c.bdir.as<float2>();
    a.act = c.bact.as<int>();
    a.obs = c.bobs.as<double>();
    a.N = N;
    a.ldE = bs.ldE;
    a.Nk = h.Nk;
    a.Nb = h.Nb;
    a.r = r;
    a.ldu = ldu;
    a.Bp = Bp;
    a.B = B;
    a.mode = TDAGW_LOWRANK;
    a.kahan = (flags & TDAGW_FLAG_NO_KAHAN) ? 0 : 1;
    a.c1 = h.c1;
    for (int q = 0; q < 4; ++q) a.occ[q] = (float)h.occ[q];
    a.dt = (float)dt;
    a.wait_ns = 2000000000ull;
    c.sync.ensure(4 * sizeof(unsigned));
    a.bar = reinterpret_cast<unsigned long long*>(c.sync.p);
    a.err = reinterpret_cast<int*>(c.sync.as<unsigned>() + 2);
    a.Rg = plan.Rg;
    a.Tg = plan.Tg;
    a.Tmax = bs.Tmax;
    c.bP.ensure((size_t)std::max(1, plan.Rg * std::max(r, 1)) * Bp * sizeof(float2));
    c.bY.ensure((size_t)std::max(r, 1) * Bp * sizeof(float2));
    c.bred.ensure((size_t)plan.Rg * Bp * 3 * sizeof(double));
    a.P = c.bP.as<float2>();
    a.Y = c.bY.as<float2>();
    a.red = c.bred.as<double>();
    AdjointState& st = c.adj;
    st = AdjointState{};
    st.valid = true;
    st.B = B;
    st.Bp = Bp;
    st.Tmax = bs.Tmax;
    st.Rg = plan.Rg;
    st.Tg = plan.Tg;
    st.mode = TDAGW_LOWRANK;
    st.dt = dt;
    st.perm = bs.perm;
    st.steps.assign(steps, steps + B);
    st.fields.assign(fields, fields + B);
    for (tdagw_field& f : st.fields) f.table = nullptr;
    st.fwd_args.resize(sizeof(BatchArgs));
    std::memcpy(st.fwd_args.data(), &a, sizeof(BatchArgs));
    st.fwd_fn = fn;
}

}  // namespace tdagw
