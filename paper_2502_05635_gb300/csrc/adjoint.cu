// Exact discrete adjoint of the batched RK4 propagation of Eq. tdagw (complex64):
// gradients of an objective of the recorded observables (P, J and occupation, Sec. "SVD
// acceleration of TD-aGW") with respect to the per-trajectory field samples E(j dt/2) (and,
// on the host, the pulse parameters).  The paper differentiates nothing; the kernel term
// is the transpose of Eq. sigma-from-k / Eq. svd_acc.
//
// With the real inner product <a, b> = Re sum conj(a_i) b_i and lam = dJ/dx_{n+1}, one RK4
// step is reversed stage by stage (stage inputs X_s and dSigma_s = K X_s recorded by a
// forward recompute of the step's segment):
//   g4 = h/6 lam,            mu4 = VJP_4(g4)
//   g3 = h/3 lam + h mu4,    mu3 = VJP_3(g3)
//   g2 = h/3 lam + h/2 mu3,  mu2 = VJP_2(g2)
//   g1 = h/6 lam + h/2 mu2,  mu1 = VJP_1(g1)
//   dJ/dx_n = lam + mu1 + mu2 + mu3 + mu4 + (direct terms of the observables at n)
// with, per k block, for f(X) = -i [A, rho], A = diag(eps) + E D + dSigma, rho = rho0 + X:
//   VJP(g) = i (A^+ g - g A^+) + K^H [ i (g rho^+ - rho^+ g) ],   Ebar = <g, -i [D, rho]>.
// K^H = conj(K^diag) + V diag(S) U^H for the low-rank factors (with the k-block reading of
// K^diag, its blocks conjugate-transposed); the dense kernel of the
// model is exactly Hermitian (its builder evaluates each entry and its transpose as exact
// conjugates), so K^H = K there.  The K^H products use the same block decomposition and
// register-tiled products as the forward kernel (U and V exchange roles).
//
// Checkpointing: the forward run stores the compensated state every C = ceil(sqrt(T))
// steps; the backward sweep recomputes one segment of C steps at a time (recording stage
// inputs) and reverses it -- memory O(sqrt(T) N B), cost about three forward runs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batched_common.cuh"

namespace tdagw {

using namespace batched;

namespace {

struct AdjArgs {
    BatchArgs b;          // model, factors, partition, barrier words (b.X etc. unused)
    const float2* recX;   // [step * 4 + stage][N][Bp] stage inputs of this segment
    const float2* recDS;  // same layout: dSigma of each stage
    float2* lam;          // dJ/dx (N x Bp)
    float2* mu;           // VJP of the previous (later) stage
    float2* musum;        // sum of the stage VJPs of this step
    float2* c1;           // local part i (A^+ g - g A^+)
    float2* mm;           // i (g rho^+ - rho^+ g), the operand of K^H
    float2* khm;          // K^H mm
    const float2* diagc;  // conj(K^diag)
    const double* dJ;     // dJ/d(observables), (Tmax + 1) x B x 3, sorted order
    double* red2;         // Rg x Bp x 4 partial Ebar per stage
    double* gE;           // B x ldE: dJ/dE_j (sorted order)
    int seg0, seglen;
};

__device__ __forceinline__ float2 mul_i(float2 z) { return make_float2(-z.y, z.x); }

// local part of the stage VJP for one (k, trajectory) block; returns Ebar
template <int NB>
__device__ double vjp_local(const AdjArgs& a, int k, int b, int slot, float E, float2 dr, float cl,
                            float cm) {
    constexpr int NB2 = NB * NB;
    const BatchArgs& m = a.b;
    const int64_t Bp = m.Bp;
    float2 G[NB2], X[NB2], M[NB2];
    // D = dir . d of the k-point, recomputed where it is used from the (L1-resident)
    // dipoles instead of held in registers
    const float2* dxk = m.dx + (int64_t)k * NB2;
    const float2* dyk = m.dy + (int64_t)k * NB2;
    auto Dq = [&](int q) {
        const float2 d1 = __ldg(dxk + q), d2 = __ldg(dyk + q);
        return make_float2(dr.x * d1.x + dr.y * d2.x, dr.x * d1.y + dr.y * d2.y);
    };
#pragma unroll
    for (int q = 0; q < NB2; ++q) {
        const int64_t i = (int64_t)k * NB2 + q;
        const int64_t e = i * Bp + b;
        const float2 l = __ldcg(a.lam + e);
        float2 g = cscale(l, cl);
        if (cm != 0.f) g = cfma(make_float2(cm, 0.f), __ldcg(a.mu + e), g);
        G[q] = g;
        X[q] = __ldcg(a.recX + (int64_t)slot * m.N * Bp + e);
        const float2 ds = __ldcg(a.recDS + (int64_t)slot * m.N * Bp + e);
        const float2 D = Dq(q);
        M[q] = make_float2(ds.x + E * D.x, ds.y + E * D.y);
    }
    double ebar = 0.0;
#pragma unroll
    for (int n = 0; n < NB; ++n)
#pragma unroll
        for (int mm = 0; mm < NB; ++mm) {
            const int q = n * NB + mm;
            const int64_t i = (int64_t)k * NB2 + q;
            // (A^+ g - g A^+)_nm = (eps_n - eps_m) g_nm + sum_l (conj(M_ln) g_lm - g_nl conj(M_ml))
            float2 t1 = gap_times(m.gap[i], G[q]);
            // (g rho^+ - rho^+ g)_nm = g_nm (f_m - f_n) + sum_l (g_nl conj(X_ml) - conj(X_ln) g_lm)
            float2 t2 = cscale(G[q], m.occ[mm] - m.occ[n]);
            // [D, rho]_nm = D_nm (f_m - f_n) + sum_l (D_nl X_lm - X_nl D_lm)
            float2 t3 = cscale(Dq(q), m.occ[mm] - m.occ[n]);
#pragma unroll
            for (int l = 0; l < NB; ++l) {
                t1 = cadd(t1, cmul(cconj(M[l * NB + n]), G[l * NB + mm]));
                t1 = csub(t1, cmul(G[n * NB + l], cconj(M[mm * NB + l])));
                t2 = cadd(t2, cmul(G[n * NB + l], cconj(X[mm * NB + l])));
                t2 = csub(t2, cmul(cconj(X[l * NB + n]), G[l * NB + mm]));
                t3 = cadd(t3, cmul(Dq(n * NB + l), X[l * NB + mm]));
                t3 = csub(t3, cmul(X[n * NB + l], Dq(l * NB + mm)));
            }
            const int64_t e = i * Bp + b;
            a.c1[e] = mul_i(t1);
            a.mm[e] = mul_i(t2);
            // Re conj(g) (-i t3) = Re(g) Im(t3) - Im(g) Re(t3)
            ebar += (double)G[q].x * (double)t3.y - (double)G[q].y * (double)t3.x;
        }
    return ebar;
}

template <int NB>
__global__ void __launch_bounds__(kBThreads, 1) adjoint_kernel(AdjArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    float2* sA = sm;
    float2* sB = sA + kChunk * kLdA;
    double* sred = reinterpret_cast<double*>(sA + kGemmSmem);
    __shared__ int abort_s;
    const BatchArgs& m = a.b;
    const int tid = threadIdx.x;
    const int rg = blockIdx.x % m.Rg, tg = blockIdx.x / m.Rg;
    const int ka = (int)((int64_t)rg * m.Nk / m.Rg), kb = (int)((int64_t)(rg + 1) * m.Nk / m.Rg);
    const int NB2 = NB * NB;
    const int64_t ra = (int64_t)ka * NB2;
    const int nrows = (kb - ka) * NB2;
    const int jr0 = (int)((int64_t)rg * m.r / m.Rg), jr1 = (int)((int64_t)(rg + 1) * m.r / m.Rg);
    const float h = m.dt;
    const float cls[4] = {h / 6.f, h / 3.f, h / 3.f, h / 6.f};  // coefficient of lam, stage s
    const float cms[4] = {0.5f * h, 0.5f * h, h, 0.f};          // coefficient of mu_{s+1}
    if (tid == 0) abort_s = 0;
    __syncthreads();
    unsigned gen = 0;
    bool ok = true;
    int prev_act = -1;
    for (int nl = a.seglen - 1; nl >= 0 && ok; --nl) {
        const int n = a.seg0 + nl;
        const int Bact = m.act[n];
        int b0, b1;
        group_range(Bact, m.Tg, tg, b0, b1);
        const int nb = b1 - b0;
        if (prev_act >= 0 && Bact != prev_act && !(ok = bgrid_sync(m, gen, &abort_s))) break;
        prev_act = Bact;
        for (int s = 3; s >= 0 && ok; --s) {
            const int eoff = s == 0 ? 0 : (s == 3 ? 2 : 1);
            // local part (own rows, own trajectories), Ebar partial per trajectory
            {
                const int bl = tid % kTileB, kg = tid / kTileB;
                double eb = 0.0;
                if (bl < nb) {
                    const int b = b0 + bl;
                    const float E = (float)m.Etab[(int64_t)b * m.ldE + 2 * n + eoff];
                    const float2 dr = m.dir[b];
                    for (int k = ka + kg; k < kb; k += kBThreads / kTileB)
                        eb += vjp_local<NB>(a, k, b, nl * 4 + s, E, dr, cls[s], cms[s]);
                }
                sred[kg * kTileB + bl] = eb;
            }
            __syncthreads();
            for (int bl = tid; bl < nb; bl += kBThreads) {
                double eb = 0.0;
                for (int kg = 0; kg < kBThreads / kTileB; ++kg) eb += sred[kg * kTileB + bl];
                a.red2[((int64_t)rg * m.Bp + b0 + bl) * 4 + s] = eb;
            }
            if (m.mode == TDAGW_LOWRANK) {
                if (nb > 0)
                    block_gemm<true>(m.U + ra * m.ldu, m.ldu, m.r, nrows, a.mm + ra * m.Bp + b0, m.Bp, nb,
                                     m.P + (int64_t)rg * m.r * m.Bp + b0, m.Bp, false, nullptr, nullptr, sA, sB);
                if (!(ok = bgrid_sync(m, gen, &abort_s))) break;
            } else {
                if (!(ok = bgrid_sync(m, gen, &abort_s))) break;
            }
            // dJ/dE at this stage's sample: sum of the row-group partials
            if (rg == 0)
                for (int b = b0 + tid; b < b1; b += kBThreads) {
                    double eb = 0.0;
                    for (int g2 = 0; g2 < m.Rg; ++g2) eb += __ldcg(a.red2 + ((int64_t)g2 * m.Bp + b) * 4 + s);
                    a.gE[(int64_t)b * m.ldE + 2 * n + eoff] += eb;
                }
            if (m.mode == TDAGW_LOWRANK) {
                for (int e = tid; e < (jr1 - jr0) * nb; e += kBThreads) {
                    const int j = jr0 + e / nb, b = b0 + e % nb;
                    float2 sum = make_float2(0.f, 0.f);
                    for (int g2 = 0; g2 < m.Rg; ++g2)
                        sum = cadd(sum, __ldcg(m.P + ((int64_t)g2 * m.r + j) * m.Bp + b));
                    m.Y[(int64_t)j * m.Bp + b] = cscale(sum, m.S[j]);
                }
                if (!(ok = bgrid_sync(m, gen, &abort_s))) break;
                if (nb > 0)
                    block_gemm<false>(m.V + ra * m.ldu, m.ldu, nrows, m.r, m.Y + b0, m.Bp, nb,
                                      a.khm + ra * m.Bp + b0, m.Bp, m.kblk == nullptr, a.diagc + ra,
                                      a.mm + ra * m.Bp + b0, sA, sB);
                if (m.kblk) {  // K^H: the conjugate-transposed k = k' blocks
                    __syncthreads();
                    if (nb > 0) kblock_term<NB, true>(m.kblk, a.mm, a.khm, m.Bp, ra, nrows, b0, nb);
                }
            } else {
                if (nb > 0)
                    block_gemm<false>(m.K + ra * m.N, m.N, nrows, (int)m.N, a.mm + b0, m.Bp, nb,
                                      a.khm + ra * m.Bp + b0, m.Bp, false, nullptr, nullptr, sA, sB);
                // all rows of mm are read before the next stage rewrites them
                if (!(ok = bgrid_sync(m, gen, &abort_s))) break;
            }
            __syncthreads();
            // mu_s = c1 + K^H mm; accumulate the step's sum
            for (int e = tid; e < nrows * nb; e += kBThreads) {
                const int64_t off = (ra + e / nb) * m.Bp + b0 + e % nb;
                const float2 mu = cadd(__ldcg(a.c1 + off), __ldcg(a.khm + off));
                a.mu[off] = mu;
                a.musum[off] = s == 3 ? mu : cadd(__ldcg(a.musum + off), mu);
            }
            __syncthreads();
        }
        if (!ok) break;
        // lam <- lam + sum of stage VJPs + direct terms of the observables at step n
        const double inv = 1.0 / (double)m.Nk;
        for (int e = tid; e < nrows * nb; e += kBThreads) {
            const int64_t i = ra + e / nb;
            const int b = b0 + e % nb;
            const int64_t off = i * m.Bp + b;
            const double* dj = a.dJ + ((int64_t)n * m.B + b) * 3;
            const float2 d1 = m.dx[i], v1 = m.vx[i];
            const int q = (int)(i % NB2);
            const float wP = (float)(dj[0] * inv), wJ = (float)(dj[1] * inv);
            const float wo = (q / NB == m.c1 && q % NB == m.c1) ? (float)(dj[2] * inv) : 0.f;
            float2 l = cadd(__ldcg(a.lam + off), __ldcg(a.musum + off));
            l = make_float2(l.x + wP * d1.x + wJ * v1.x + wo, l.y + wP * d1.y + wJ * v1.y);
            a.lam[off] = l;
        }
        __syncthreads();
    }
}

__global__ void ck_restore_kernel(const float2* __restrict__ ckS, const float2* __restrict__ ckC,
                                  float2* __restrict__ S, float2* __restrict__ C, float2* __restrict__ X,
                                  int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 s = ckS[e], c = ckC[e];
        S[e] = s;
        C[e] = c;
        X[e] = cadd(s, c);
    }
}

// lam = direct terms at each trajectory's final step T_b
__global__ void lam_init_kernel(float2* __restrict__ lam, const float2* __restrict__ dx,
                                const float2* __restrict__ vx, const double* __restrict__ dJ,
                                const int* __restrict__ Tsorted, int64_t N, int Nb, int c1, int B, int Bp,
                                int Nk) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * Bp) return;
    const int64_t i = e / Bp;
    const int b = (int)(e % Bp);
    float2 l = make_float2(0.f, 0.f);
    if (b < B) {
        const double* dj = dJ + ((int64_t)Tsorted[b] * B + b) * 3;
        const double inv = 1.0 / Nk;
        const int q = (int)(i % (Nb * Nb));
        const float wP = (float)(dj[0] * inv), wJ = (float)(dj[1] * inv);
        const float wo = (q / Nb == c1 && q % Nb == c1) ? (float)(dj[2] * inv) : 0.f;
        l = make_float2(wP * dx[i].x + wJ * vx[i].x + wo, wP * dx[i].y + wJ * vx[i].y);
    }
    lam[e] = l;
}

__global__ void conj_kernel(const float2* __restrict__ src, float2* __restrict__ dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = cconj(src[e]);
}

}  // namespace

// Backward sweep over the last checkpointed batched propagation (see the file comment).
// dJdobs: host (Tmax + 1) x B x 3; dJdE: host (2 Tmax + 1) x B; dJdparams: host B x 4 or NULL.
void adjoint_batched(Ctx& c, const double* dJdobs, double* dJdE, double* dJdparams) {
    AdjointState& st = c.adj;
    TDAGW_REQUIRE(st.valid, TDAGW_ERR_INVALID_ARG,
                  "tdagw_adjoint needs a preceding tdagw_propagate with TDAGW_FLAG_CHECKPOINT");
    const HostModel& h = c.hm;
    cudaStream_t s = c.stream;
    const int B = st.B, Bp = st.Bp, Tmax = st.Tmax, C = st.period;
    const int64_t N = h.N, ldE = 2 * (int64_t)Tmax + 1;
    // objective derivatives in sorted trajectory order
    std::vector<double> dj((size_t)(Tmax + 1) * B * 3);
    for (int n = 0; n <= Tmax; ++n)
        for (int q = 0; q < B; ++q)
            for (int z = 0; z < 3; ++z) {
                const int b = st.perm[q];
                const double v = n <= st.steps[b] ? dJdobs[((int64_t)n * B + b) * 3 + z] : 0.0;
                dj[((size_t)n * B + q) * 3 + z] = std::isfinite(v) ? v : 0.0;
            }
    DevBuf ddj, dT, gE, red2, diagc;
    ddj.ensure(dj.size() * sizeof(double));
    TDAGW_CUDA(cudaMemcpyAsync(ddj.p, dj.data(), dj.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    std::vector<int> Ts(B);
    for (int q = 0; q < B; ++q) Ts[q] = st.steps[st.perm[q]];
    dT.ensure(B * sizeof(int));
    TDAGW_CUDA(cudaMemcpyAsync(dT.p, Ts.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    gE.ensure((size_t)B * ldE * sizeof(double));
    TDAGW_CUDA(cudaMemsetAsync(gE.p, 0, (size_t)B * ldE * sizeof(double), s));
    red2.ensure((size_t)st.Rg * Bp * 4 * sizeof(double));
    const size_t sb = (size_t)N * Bp * sizeof(float2);
    for (DevBuf* b : {&c.aLam, &c.aMu, &c.aMusum, &c.aC1, &c.aMm, &c.aKhm}) b->ensure(sb);
    const int64_t rec_slots = 4 * (int64_t)C;
    c.aRecX.ensure((size_t)rec_slots * sb);
    c.aRecDS.ensure((size_t)rec_slots * sb);
    if (st.mode == TDAGW_LOWRANK) {
        diagc.ensure(N * sizeof(float2));
        conj_kernel<<<152 * 4, 256, 0, s>>>(c.diagF.as<float2>(), diagc.as<float2>(), N);
        check_launch("conj_kernel");
    }
    lam_init_kernel<<<(unsigned)((N * Bp + 255) / 256), 256, 0, s>>>(
        c.aLam.as<float2>(), c.dx.as<float2>(), c.vx.as<float2>(), ddj.as<double>(), dT.as<int>(), N, h.Nb,
        h.c1, B, Bp, h.Nk);
    check_launch("lam_init_kernel");

    // forward-recompute launch parameters (records on, checkpoints off, scratch observables)
    BatchArgs fa;
    std::memcpy(&fa, st.fwd_args.data(), sizeof(BatchArgs));
    DevBuf scratch_obs;
    scratch_obs.ensure((size_t)(C + 1) * B * 3 * sizeof(double));
    fa.obs = scratch_obs.as<double>();
    fa.ckS = nullptr;
    fa.ckC = nullptr;
    fa.recX = c.aRecX.as<float2>();
    fa.recDS = c.aRecDS.as<float2>();
    AdjArgs aa{};
    aa.b = fa;
    aa.recX = c.aRecX.as<float2>();
    aa.recDS = c.aRecDS.as<float2>();
    aa.lam = c.aLam.as<float2>();
    aa.mu = c.aMu.as<float2>();
    aa.musum = c.aMusum.as<float2>();
    aa.c1 = c.aC1.as<float2>();
    aa.mm = c.aMm.as<float2>();
    aa.khm = c.aKhm.as<float2>();
    aa.diagc = diagc.as<float2>();
    aa.dJ = ddj.as<double>();
    aa.red2 = red2.as<double>();
    aa.gE = gE.as<double>();
    const size_t smem = (size_t)kGemmSmem * sizeof(float2) +
                        (size_t)(kBThreads / kTileB) * kTileB * 3 * sizeof(double);
    const void* ffn = st.fwd_fn;
    const void* bfn = h.Nb == 2 ? (const void*)adjoint_kernel<2> : (const void*)adjoint_kernel<4>;
    TDAGW_CUDA(cudaFuncSetAttribute(bfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grid(st.Rg * st.Tg);
    const int nseg = (Tmax + C - 1) / C;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int n0 = sg * C, len = std::min(C, Tmax - n0);
        const int64_t slot = (int64_t)sg * N * Bp;
        ck_restore_kernel<<<152 * 4, 256, 0, s>>>(c.ckS.as<float2>() + slot, c.ckC.as<float2>() + slot,
                                                  c.bS.as<float2>(), c.bC.as<float2>(), c.bX.as<float2>(), N * Bp);
        check_launch("ck_restore_kernel");
        if (st.tc) {
            // the forward ran on the tensor cores: recompute the segment there too
            tc_recompute_segment(c, n0, len, fa.recX, fa.recDS, fa.obs);
        } else {
            fa.n0 = n0;
            fa.Tmax = len;
            TDAGW_CUDA(cudaMemsetAsync(c.sync.p, 0, 4 * sizeof(unsigned), s));
            void* fargs[] = {&fa};
            TDAGW_CUDA(cudaLaunchCooperativeKernel(ffn, grid, dim3(kBThreads), fargs, smem, s));
        }
        aa.seg0 = n0;
        aa.seglen = len;
        TDAGW_CUDA(cudaMemsetAsync(c.sync.p, 0, 4 * sizeof(unsigned), s));
        void* bargs[] = {&aa};
        TDAGW_CUDA(cudaLaunchCooperativeKernel(bfn, grid, dim3(kBThreads), bargs, smem, s));
        c.persistent_launched = true;
    }
    std::vector<double> hg((size_t)B * ldE);
    TDAGW_CUDA(cudaMemcpyAsync(hg.data(), gE.p, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
    int err = 0;
    TDAGW_CUDA(cudaMemcpy(&err, c.sync.as<unsigned>() + 2, sizeof(int), cudaMemcpyDeviceToHost));
    TDAGW_REQUIRE(!err, TDAGW_ERR_TIMEOUT, "a bounded device-side wait of the adjoint gave up");
    const double dt = st.dt;
    for (int q = 0; q < B; ++q) {
        const int b = st.perm[q];
        const tdagw_field& f = st.fields[b];
        double gp[4] = {0, 0, 0, 0};
        for (int64_t j = 0; j < ldE; ++j) {
            const double g = j <= 2 * (int64_t)st.steps[b] ? hg[(size_t)q * ldE + j] : 0.0;
            if (dJdE) dJdE[j * B + b] = g;
            if (f.kind == TDAGW_FIELD_GAUSS_COS && g != 0.0) {
                // dE/d(E0, omega, t0, sigma) of E0 exp(-(t - t0)^2 / (2 sigma^2)) cos(omega t)
                const double t = 0.5 * dt * (double)j, u = t - f.t0;
                const double env = std::exp(-(u * u) / (2.0 * f.sigma * f.sigma));
                const double cs = std::cos(f.omega * t), sn = std::sin(f.omega * t);
                const double E = f.E0 * env * cs;
                gp[0] += g * env * cs;
                gp[1] += g * (-f.E0 * env * t * sn);
                gp[2] += g * E * u / (f.sigma * f.sigma);
                gp[3] += g * E * u * u / (f.sigma * f.sigma * f.sigma);
            }
        }
        if (dJdparams)
            for (int z = 0; z < 4; ++z) dJdparams[(int64_t)b * 4 + z] = gp[z];
    }
}

}  // namespace tdagw
