// Per-stage kernels of the propagation: the kernel contraction dSigma = K . X as a
// streaming complex GEMV (dense form of Eq. sigma-from-k, and the two passes of the
// truncated-SVD form of Eq. svd_acc), and the fused per-k commutator + RK4 stage update +
// observables kernel (Eq. tdagw).
#include "common.cuh"
#include "stage.cuh"

namespace tdagw {

namespace {

// ---------------------------------------------------------------- vector loads -------

// Two consecutive complex elements; streaming (evict-first) loads for matrix operands
// that are read once per stage, cached loads for the vector operand.
__device__ __forceinline__ void ld2_stream(const float2* p, float2& a, float2& b) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld2_stream(const double2* p, double2& a, double2& b) {
    a = __ldcs(p);
    b = __ldcs(p + 1);
}
__device__ __forceinline__ void ld2_cached(const float2* p, float2& a, float2& b) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld2_cached(const double2* p, double2& a, double2& b) {
    a = __ldg(p);
    b = __ldg(p + 1);
}

// ---------------------------------------------------------------- GEMV ---------------

// out[row] = sum_c A[row, c] x[c] (+ diag[row] xd[row]) for ROWS rows per block.  Each
// thread walks the block's column range two complex at a time (16 B per row per step for
// c64) so that a warp covers 512 contiguous bytes of each row per load; the ROWS
// accumulators share every load of x.  nsplit > 1 splits the columns into nsplit ranges
// and writes nsplit partial vectors (split-K) instead.
template <typename R, int ROWS, int THREADS>
__global__ void __launch_bounds__(THREADS)
gemv_kernel(const cplx_t<R>* __restrict__ A, int64_t lda, int64_t nrows, int64_t ncols,
            const cplx_t<R>* __restrict__ x, cplx_t<R>* __restrict__ out, int nsplit,
            const cplx_t<R>* __restrict__ diag, const cplx_t<R>* __restrict__ xd) {
    using C = cplx_t<R>;
    const int64_t rg = blockIdx.x / nsplit;
    const int split = blockIdx.x % nsplit;
    const int64_t r0 = rg * ROWS;
    int64_t cs = (ncols + nsplit - 1) / nsplit;
    cs += cs & 1;
    const int64_t c0 = split * cs;
    const int64_t c1 = min(ncols, c0 + cs);
    C acc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r] = mk((R)0, (R)0);
    const int tid = threadIdx.x;
    bool valid[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) valid[r] = (r0 + r) < nrows;

    int64_t c = c0 + 2 * tid;
#pragma unroll 2
    for (; c + 1 < c1; c += 2 * THREADS) {
        C x0, x1;
        ld2_cached(x + c, x0, x1);
        C a0[ROWS], a1[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (valid[r]) ld2_stream(A + (r0 + r) * lda + c, a0[r], a1[r]);
            else a0[r] = a1[r] = mk((R)0, (R)0);
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) acc[r] = cfma(a1[r], x1, cfma(a0[r], x0, acc[r]));
    }
    if (c1 > c0 && ((c1 - c0) & 1) && tid == 0) {
        const int64_t cl = c1 - 1;
        const C xl = x[cl];
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
            if (valid[r]) acc[r] = cfma(A[(r0 + r) * lda + cl], xl, acc[r]);
    }
    // block reduction: warp shuffles, then across warps in shared memory
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[r] = cadd(acc[r], shfl_xor(acc[r], o));
    constexpr int NW = THREADS / 32;
    __shared__ C red[NW][ROWS];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int r = 0; r < ROWS; ++r) red[warp][r] = acc[r];
    __syncthreads();
    if (tid < ROWS && valid[tid]) {
        C s = red[0][tid];
#pragma unroll
        for (int w = 1; w < NW; ++w) s = cadd(s, red[w][tid]);
        const int64_t row = r0 + tid;
        if (nsplit == 1) {
            if (diag) s = cfma(diag[row], xd[row], s);
            out[row] = s;
        } else {
            out[(int64_t)split * nrows + row] = s;
        }
    }
}

// y = V^H x with V stored N x ldu row-major: block (b, cb) accumulates
//   part[b][c] = sum_{i in rows of b} conj(V[i][c]) x_i
// for its 512 columns c (two per thread), streaming the rows of V (16 B per thread per
// row, so a warp reads 256 contiguous bytes).
template <typename R>
__global__ void __launch_bounds__(256)
vcols_kernel(const cplx_t<R>* __restrict__ V, int64_t ldv, int64_t N, int r,
             const cplx_t<R>* __restrict__ x, cplx_t<R>* __restrict__ part, int64_t rpb) {
    using C = cplx_t<R>;
    const int64_t i0 = blockIdx.x * rpb, i1 = min(N, i0 + rpb);
    const int64_t c = (int64_t)blockIdx.y * 512 + 2 * threadIdx.x;
    if (c >= ldv) return;
    C a0 = mk((R)0, (R)0), a1 = a0;
#pragma unroll 4
    for (int64_t i = i0; i < i1; ++i) {
        C v0, v1;
        ld2_stream(V + i * ldv + c, v0, v1);
        const C xi = __ldg(x + i);
        a0 = cfmac(v0, xi, a0);
        a1 = cfmac(v1, xi, a1);
    }
    if (c < r) part[(int64_t)blockIdx.x * r + c] = a0;
    if (c + 1 < r) part[(int64_t)blockIdx.x * r + c + 1] = a1;
}

// ytil[j] = S[j] * sum_s part[s][j]: finishes y = S o (V^H x) of Eq. svd_acc.
template <typename R>
__global__ void yreduce_kernel(const cplx_t<R>* __restrict__ part, int nsplit, int r,
                               const R* __restrict__ S, cplx_t<R>* __restrict__ ytil) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= r) return;
    cplx_t<R> s = part[j];
    for (int q = 1; q < nsplit; ++q) s = cadd(s, part[(int64_t)q * r + j]);
    ytil[j] = cscale(s, S[j]);
}

// ---------------------------------------------------------------- stage --------------

// Block partial sums of (P_x, J_x, occ_c1) in FP64, then the last block to arrive adds
// the partials in block order (deterministic) and stores row `row` of obs.
__device__ void reduce_observables(double v0, double v1, double v2, double* red,
                                   unsigned* counter, double* obs_row, double inv_nk,
                                   int64_t* step_to_bump, int64_t new_step) {
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    __shared__ double sred[32][3];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sred[warp][0] = v0;
        sred[warp][1] = v1;
        sred[warp][2] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sred[w][0];
            b += sred[w][1];
            c += sred[w][2];
        }
        red[blockIdx.x * 3 + 0] = a;
        red[blockIdx.x * 3 + 1] = b;
        red[blockIdx.x * 3 + 2] = c;
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double a = 0, b = 0, c = 0;
        for (unsigned q = 0; q < gridDim.x; ++q) {
            a += ((volatile double*)red)[q * 3 + 0];
            b += ((volatile double*)red)[q * 3 + 1];
            c += ((volatile double*)red)[q * 3 + 2];
        }
        obs_row[0] = a * inv_nk;
        obs_row[1] = b * inv_nk;
        obs_row[2] = c * inv_nk;
        *counter = 0u;
        if (step_to_bump) *step_to_bump = new_step;
    }
}

// One RK4 stage for all k: k_s = -i [diag(eps) + E(t_s).d + dSigma, rho0 + X_s] per k
// (Eq. tdagw with dSigma from Eq. sigma-from-k), accumulated into the classical RK4
// combination; the next stage input X_{s+1} = drho_n + c_{s+1} dt k_s is written directly.
// On the last stage the state is advanced with a compensated (TwoSum) accumulation and
// the observables of the new state are reduced.  One thread per pair element (k, n, m);
// the Nb^2 threads of one k are adjacent lanes of a warp and exchange the Nb x Nb blocks
// by shuffles.
template <typename R, int NB>
__global__ void __launch_bounds__(256) stage_kernel(StageParams<R> p) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nstep = *p.step;
    const int eoff = p.stage == 0 ? 0 : (p.stage == 3 ? 2 : 1);
    const R E = (R)p.Etab[2 * nstep + eoff];
    Obs3 ob{0.0, 0.0, 0.0};
    stage_element<R, NB>(p, i, i < p.N, threadIdx.x & 31, p.stage, E, ob);
    if (p.stage == 3)
        reduce_observables(ob.p, ob.j, ob.o, p.red, p.counter, p.obs + (nstep + 1) * 3,
                           1.0 / (double)p.Nk, p.step, nstep + 1);
}

// Observables of rho0 + X into obs row `row` (used for the initial row of a run).
template <typename R, int NB>
__global__ void __launch_bounds__(256)
observables_kernel(const cplx_t<R>* __restrict__ X, const cplx_t<R>* __restrict__ dx,
                   const cplx_t<R>* __restrict__ vx, int64_t N, int Nk, int c1, R o0_, R o1_,
                   R o2_, R o3_, double* red, unsigned* counter, double* obs_row) {
    using C = cplx_t<R>;
    constexpr int NB2 = NB * NB;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int g = (threadIdx.x & 31) % NB2, n = g / NB, m = g % NB;
    const R occ[4] = {o0_, o1_, o2_, o3_};
    double a = 0, b = 0, c = 0;
    if (i < N) {
        C rho = X[i];
        if (n == m) rho.x += occ[n];
        const C d = dx[i], v = vx[i];
        a = (double)rho.x * (double)d.x + (double)rho.y * (double)d.y;
        b = (double)rho.x * (double)v.x + (double)rho.y * (double)v.y;
        c = (n == m && n == c1) ? (double)rho.x : 0.0;
    }
    reduce_observables(a, b, c, red, counter, obs_row, 1.0 / (double)Nk, nullptr, 0);
}

// the k = k' blocks of K: out[(k P + p) P + q] = K[(k P + p) N + k P + q]
template <typename R>
__global__ void gather_kblocks_kernel(const cplx_t<R>* __restrict__ K, int64_t N, int Nk, int P,
                                      cplx_t<R>* __restrict__ out) {
    const int64_t n = (int64_t)Nk * P * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / (P * P), r = e % (P * P);
        const int p = (int)(r / P), q = (int)(r % P);
        out[e] = K[(k * P + p) * N + k * P + q];
    }
}

// y[k P + p] += sum_q B[k][p][q] x[k P + q]: the k-block reading of K^diag x
template <typename R>
__global__ void kblock_add_kernel(const cplx_t<R>* __restrict__ B, const cplx_t<R>* __restrict__ x,
                                  cplx_t<R>* __restrict__ y, int Nk, int P) {
    using C = cplx_t<R>;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)Nk * P) return;
    const int64_t k = i / P;
    const int p = (int)(i % P);
    const C* b = B + (k * P + p) * P;
    const C* xk = x + k * P;
    C s = y[i];
    for (int q = 0; q < P; ++q) s = cfma(b[q], xk[q], s);
    y[i] = s;
}

}  // namespace

template <typename R>
void launch_gather_kblocks(const Ctx& c, void* dst, cudaStream_t s) {
    const HostModel& h = c.hm;
    gather_kblocks_kernel<R><<<152 * 4, 256, 0, s>>>(c.K.as<cplx_t<R>>(), h.N, h.Nk, h.Nb * h.Nb,
                                                     static_cast<cplx_t<R>*>(dst));
    check_launch("gather_kblocks_kernel");
}

template <typename R>
void launch_kblock_add(const void* B, const void* x, void* y, int Nk, int P, cudaStream_t s) {
    using C = cplx_t<R>;
    const int64_t n = (int64_t)Nk * P;
    kblock_add_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        static_cast<const C*>(B), static_cast<const C*>(x), static_cast<C*>(y), Nk, P);
    check_launch("kblock_add_kernel");
}

template <typename R>
void launch_gemv(const void* A, int64_t lda, int64_t nrows, int64_t ncols, const void* x,
                 void* out, int nsplit, const void* diag, const void* xd, cudaStream_t s) {
    using C = cplx_t<R>;
    constexpr int ROWS = 4, THREADS = 256;
    const int64_t rgs = (nrows + ROWS - 1) / ROWS;
    const int64_t blocks = rgs * nsplit;
    gemv_kernel<R, ROWS, THREADS><<<(unsigned)blocks, THREADS, 0, s>>>(
        static_cast<const C*>(A), lda, nrows, ncols, static_cast<const C*>(x),
        static_cast<C*>(out), nsplit, static_cast<const C*>(diag), static_cast<const C*>(xd));
    check_launch("gemv_kernel");
}

template <typename R>
void launch_vcols(const void* V, int64_t ldv, int64_t N, int r, const void* x, void* part,
                  int nblocks, cudaStream_t s) {
    using C = cplx_t<R>;
    const int64_t rpb = (N + nblocks - 1) / nblocks;
    dim3 grid((unsigned)nblocks, (unsigned)((ldv + 511) / 512));
    vcols_kernel<R><<<grid, 256, 0, s>>>(static_cast<const C*>(V), ldv, N, r,
                                          static_cast<const C*>(x), static_cast<C*>(part), rpb);
    check_launch("vcols_kernel");
}

template <typename R>
void launch_yreduce(const void* part, int nsplit, int r, const void* S, void* ytil,
                    cudaStream_t s) {
    using C = cplx_t<R>;
    yreduce_kernel<R><<<(r + 255) / 256, 256, 0, s>>>(static_cast<const C*>(part), nsplit, r,
                                                       static_cast<const R*>(S),
                                                       static_cast<C*>(ytil));
    check_launch("yreduce_kernel");
}

template <typename R>
void launch_stage(Ctx& c, int stage, double dt, double dirx, double diry, bool kahan,
                  cudaStream_t s) {
    using C = cplx_t<R>;
    StageParams<R> p;
    p.X = c.X.as<C>();
    p.dS = c.dS.as<C>();
    p.dx = c.dx.as<C>();
    p.dy = c.dy.as<C>();
    p.vx = c.vx.as<C>();
    p.gap = c.gap.as<typename GapT<R>::type>();
    p.acc = c.acc.as<C>();
    p.Ssum = c.Ssum.as<C>();
    p.Ccomp = c.Ccomp.as<C>();
    p.Xnext = c.X.as<C>();  // in place: each thread reads X[i] before writing it
    p.Etab = c.Etab.as<double>();
    p.step = c.stepctr.as<int64_t>();
    p.obs = c.obs.as<double>();
    p.red = c.red.as<double>();
    p.counter = c.counter.as<unsigned>();
    p.N = c.hm.N;
    p.Nk = c.hm.Nk;
    p.c1 = c.hm.c1;
    for (int q = 0; q < 4; ++q) p.occ[q] = (R)c.hm.occ[q];
    p.dt = (R)dt;
    p.dirx = (R)dirx;
    p.diry = (R)diry;
    p.stage = stage;
    p.kahan = kahan ? 1 : 0;
    const unsigned blocks = (unsigned)((c.hm.N + 255) / 256);
    if (c.hm.Nb == 2) stage_kernel<R, 2><<<blocks, 256, 0, s>>>(p);
    else stage_kernel<R, 4><<<blocks, 256, 0, s>>>(p);
    check_launch("stage_kernel");
}

template <typename R>
void launch_observables_row(Ctx& c, const void* X, int64_t row, cudaStream_t s) {
    using C = cplx_t<R>;
    const unsigned blocks = (unsigned)((c.hm.N + 255) / 256);
    const HostModel& h = c.hm;
    double* orow = c.obs.as<double>() + row * 3;
    if (h.Nb == 2)
        observables_kernel<R, 2><<<blocks, 256, 0, s>>>(
            static_cast<const C*>(X), c.dx.as<C>(), c.vx.as<C>(), h.N, h.Nk, h.c1, (R)h.occ[0],
            (R)h.occ[1], (R)h.occ[2], (R)h.occ[3], c.red.as<double>(), c.counter.as<unsigned>(), orow);
    else
        observables_kernel<R, 4><<<blocks, 256, 0, s>>>(
            static_cast<const C*>(X), c.dx.as<C>(), c.vx.as<C>(), h.N, h.Nk, h.c1, (R)h.occ[0],
            (R)h.occ[1], (R)h.occ[2], (R)h.occ[3], c.red.as<double>(), c.counter.as<unsigned>(), orow);
    check_launch("observables_kernel");
}

#define INST(R)                                                                            \
    template void launch_gemv<R>(const void*, int64_t, int64_t, int64_t, const void*, void*, \
                                 int, const void*, const void*, cudaStream_t);             \
    template void launch_yreduce<R>(const void*, int, int, const void*, void*, cudaStream_t); \
    template void launch_vcols<R>(const void*, int64_t, int64_t, int, const void*, void*, int, \
                                  cudaStream_t);                                          \
    template void launch_stage<R>(Ctx&, int, double, double, double, bool, cudaStream_t);   \
    template void launch_observables_row<R>(Ctx&, const void*, int64_t, cudaStream_t);
INST(float)
INST(double)
template void launch_gather_kblocks<float>(const Ctx&, void*, cudaStream_t);
template void launch_gather_kblocks<double>(const Ctx&, void*, cudaStream_t);
template void launch_kblock_add<float>(const void*, const void*, void*, int, int, cudaStream_t);
template void launch_kblock_add<double>(const void*, const void*, void*, int, int, cudaStream_t);
#undef INST

}  // namespace tdagw
