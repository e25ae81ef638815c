// Randomised truncated SVD of K^off = K - diag(K) on the device (setup of Eq.
// svd_diag_offdiag; with the k-block reading of K^diag, K^off = K minus its k = k' blocks).
//
// Range finder (Halko, Martinsson, Tropp 2011, randomised subspace iteration with
// re-orthonormalisation after every product):
//   Y = K^off Omega (Omega: N x l complex Gaussian, l = rank + oversample), Q = orth(Y)
//   repeat 2 * power_iters times:  Q = orth(K^off Q)
// then the SVD of B = Q^H K^off (l x N), the one-sided projection whose truncation error
// follows the HMT bounds: K^off is Hermitian, so Z = K^off Q is B^H, and
//   B B^H = Z^H Z = W diag(lambda) W^H (parallel two-sided Jacobi),
//   sigma_j = sqrt(lambda_j),  U = Q W_r,  V = Z W_r diag(1 / sigma)   (B = W Sigma V^H)
// keeping the `rank` largest.  The core squares the singular values, so sigma_j below
// 1e-7 sigma_0 is not resolved in FP64: such a triplet is kept with sigma_j = 0 (a zero V
// column) and contributes nothing.
// Products with K run in the context precision; Q, B, W and all orthogonalisation are FP64
// (block classical Gram-Schmidt with reorthogonalisation, panels of 64 columns, each panel
// made orthonormal by two Cholesky-QR passes).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace tdagw {

namespace {

// ---------------------------------------------------------------- Gaussian sketch ----

// Counter-based generator: SplitMix64 (Steele, Lea, Flood 2014) applied to seed + counter,
// two 53-bit uniforms per draw, Box-Muller to a standard complex Gaussian (unit variance).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t splitmix64_host(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gauss_kernel(double2* __restrict__ out, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix64(seed ^ splitmix64(2 * (uint64_t)i));
        const uint64_t b = splitmix64(seed ^ splitmix64(2 * (uint64_t)i + 1));
        const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);  // (0, 1]
        const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);        // [0, 1)
        const double rad = sqrt(-log(u1));                                // |z|^2 ~ Exp(1)
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        out[i] = make_double2(rad * cs, rad * sn);
    }
}

// ---------------------------------------------------------------- complex GEMM -------

template <typename R> __device__ __forceinline__ cplx_t<R> ld_as(const float2& v) {
    return mk((R)v.x, (R)v.y);
}
template <typename R> __device__ __forceinline__ cplx_t<R> ld_as(const double2& v) {
    return mk((R)v.x, (R)v.y);
}

constexpr int GBM = 64, GBN = 64, GBK = 16, GTH = 256;

// C[M x Nn] (+)= alpha op(A) op(B), op = identity or conjugate transpose (HA / HB), with
// row-major storage: op(A)[m][k] = A[m lda + k] or conj(A[k lda + m]).  Tiles of 64 x 64
// outputs, 16-deep k slices through shared memory, 4 x 4 outputs per thread; operands are
// converted to the accumulation precision Racc on load.  With ksplit > 1, block z sums
// k-range z and writes raw partials to work[z] (finished by splitk_reduce_kernel).
template <typename TA, typename TB, typename Racc, bool HA, bool HB>
__global__ void __launch_bounds__(GTH)
gemm_kernel(int M, int Nn, int K, const TA* __restrict__ A, int64_t lda, const TB* __restrict__ B,
            int64_t ldb, double2* __restrict__ C, int64_t ldc, double2 alpha, double2 beta,
            int kchunk, double2* __restrict__ work) {
    using C2 = cplx_t<Racc>;
    __shared__ C2 As[GBK][GBM + 1];
    __shared__ C2 Bs[GBK][GBN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    C2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mk((Racc)0, (Racc)0);
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        // A tile: GBM x GBK elements, 4 per thread
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * GTH;
            int mm, kk;
            if (HA) { mm = e % GBM; kk = e / GBM; } else { kk = e % GBK; mm = e / GBK; }
            const int m = m0 + mm, k = k0 + kk;
            C2 v = mk((Racc)0, (Racc)0);
            if (m < M && k < kend) {
                if (HA) v = cconj(ld_as<Racc>(A[(int64_t)k * lda + m]));
                else v = ld_as<Racc>(A[(int64_t)m * lda + k]);
            }
            As[kk][mm] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * GTH;
            int nn, kk;
            if (HB) { kk = e % GBK; nn = e / GBK; } else { nn = e % GBN; kk = e / GBN; }
            const int n = n0 + nn, k = k0 + kk;
            C2 v = mk((Racc)0, (Racc)0);
            if (n < Nn && k < kend) {
                if (HB) v = cconj(ld_as<Racc>(B[(int64_t)n * ldb + k]));
                else v = ld_as<Racc>(B[(int64_t)k * ldb + n]);
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            C2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m >= M || n >= Nn) continue;
            const double2 v = make_double2((double)acc[i][j].x, (double)acc[i][j].y);
            if (work) {
                work[((int64_t)blockIdx.z * M + m) * Nn + n] = v;
            } else {
                double2 r = cmul(alpha, v);
                if (beta.x != 0.0 || beta.y != 0.0) r = cfma(beta, C[(int64_t)m * ldc + n], r);
                C[(int64_t)m * ldc + n] = r;
            }
        }
}

__global__ void splitk_reduce_kernel(int M, int Nn, int nsplit, const double2* __restrict__ work,
                                     double2* __restrict__ C, int64_t ldc, double2 alpha,
                                     double2 beta) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * Nn) return;
    const int m = (int)(e / Nn), n = (int)(e % Nn);
    double2 s = work[e];
    for (int z = 1; z < nsplit; ++z) s = cadd(s, work[(int64_t)z * M * Nn + e]);
    double2 r = cmul(alpha, s);
    if (beta.x != 0.0 || beta.y != 0.0) r = cfma(beta, C[(int64_t)m * ldc + n], r);
    C[(int64_t)m * ldc + n] = r;
}

// Y[i][j] -= d[i] X[i][j]: removes K^diag from a product with K (K^off = K - diag K).
template <typename R>
__global__ void sub_diag_kernel(double2* __restrict__ Y, const double2* __restrict__ X, int64_t n,
                                int l, const cplx_t<R>* __restrict__ d) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * l;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / l;
        const double2 di = make_double2((double)d[i].x, (double)d[i].y);
        Y[e] = csub(Y[e], cmul(di, X[e]));
    }
}

// Y -= (k-diagonal blocks) X for X, Y (N x l, FP64, ld l): the k-block reading of K^diag
template <typename R>
__global__ void sub_kblock_kernel(double2* __restrict__ Y, const double2* __restrict__ X, int64_t N, int l,
                                  const cplx_t<R>* __restrict__ B, int P) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * l;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / l, c = e % l;
        const int64_t k = i / P;
        const int p = (int)(i % P);
        double2 s = Y[e];
        for (int q = 0; q < P; ++q) {
            const cplx_t<R> b = B[(k * P + p) * P + q];
            s = csub(s, cmul(make_double2((double)b.x, (double)b.y), X[(k * P + q) * l + c]));
        }
        Y[e] = s;
    }
}

// ---------------------------------------------------------------- small factorisations

// Given the Hermitian positive semi-definite b x b Gram matrix G (row-major, ld b), writes
// M = L^{-H} (upper triangular) for the Cholesky factor G = L L^H, so that P M has
// orthonormal columns when G = P^H P.  Tiny or negative pivots are lifted to a floor of
// 1e-13 max(diag G) so rank-deficient panels stay finite (the second pass cleans up).
// One block; b <= 64.
__global__ void chol_inv_kernel(const double2* __restrict__ G, int b, double2* __restrict__ Minv) {
    __shared__ double2 Ls[64][65];
    __shared__ double2 Zs[64][65];
    __shared__ double floor_v;
    const int t = threadIdx.x;
    for (int e = t; e < b * b; e += blockDim.x) Ls[e / b][e % b] = G[e];
    __syncthreads();
    if (t == 0) {
        double mx = 0.0;
        for (int i = 0; i < b; ++i) mx = fmax(mx, Ls[i][i].x);
        floor_v = fmax(mx * 1e-13, 1e-300);
    }
    __syncthreads();
    // left-looking Cholesky, lower factor in Ls (row i, col j <= i)
    for (int j = 0; j < b; ++j) {
        if (t == 0) {
            double s = Ls[j][j].x;
            for (int k = 0; k < j; ++k) s -= Ls[j][k].x * Ls[j][k].x + Ls[j][k].y * Ls[j][k].y;
            Ls[j][j] = make_double2(sqrt(fmax(s, floor_v)), 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / Ls[j][j].x;
        for (int i = j + 1 + t; i < b; i += blockDim.x) {
            double2 s = Ls[i][j];
            for (int k = 0; k < j; ++k) s = csub(s, cmulc(Ls[i][k], Ls[j][k]));
            Ls[i][j] = cscale(s, inv);
        }
        __syncthreads();
    }
    // Z = L^{-1} (lower), one column per thread, forward substitution
    for (int c = t; c < b; c += blockDim.x) {
        for (int i = 0; i < b; ++i) {
            if (i < c) { Zs[i][c] = make_double2(0, 0); continue; }
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int k = c; k < i; ++k) s = csub(s, cmul(Ls[i][k], Zs[k][c]));
            Zs[i][c] = cscale(s, 1.0 / Ls[i][i].x);
        }
    }
    __syncthreads();
    // M = Z^H (upper): M[i][j] = conj(Z[j][i])
    for (int e = t; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        Minv[e] = cconj(Zs[j][i]);
    }
}

// ---------------------------------------------------------------- Jacobi -------------

struct __align__(16) Rot4 {
    double x, y, z, w;  // c, s, cos phi, sin phi
};
__device__ __forceinline__ Rot4 make_rot4(double a, double b, double c, double d) {
    Rot4 r;
    r.x = a;
    r.y = b;
    r.z = c;
    r.w = d;
    return r;
}

// Round-robin ("circle") pairing of n_e (even) indices: round r, pair t.
__device__ __forceinline__ void rr_pair(int ne, int r, int t, int& p, int& q) {
    const int m = ne - 1;
    if (t == 0) { p = m; q = r; }
    else { p = (r + t) % m; q = (r - t + m) % m; }
    if (p > q) { const int x = p; p = q; q = x; }
}

// Rotation for the 2x2 Hermitian block [[a, b], [conj b, d]] at (p, q), b = |b| e^{i phi}:
// G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] zeroes the off-diagonal of G^H A G with
// t = s/c the smaller root of t^2 + 2 tau t - 1 = 0, tau = (d - a) / (2 |b|).  This kernel
// applies G^H to rows p and q (all columns) and stores (c, s, e^{i phi}).
__global__ void jacobi_rows_kernel(double2* __restrict__ A, int n, int ne, int round,
                                   Rot4* __restrict__ rot) {
    int p, q;
    rr_pair(ne, round, blockIdx.x, p, q);
    if (q >= n) return;
    __shared__ Rot4 sr;
    if (threadIdx.x == 0) {
        const double a = A[(int64_t)p * n + p].x, d = A[(int64_t)q * n + q].x;
        const double2 b = A[(int64_t)p * n + q];
        const double bb = hypot(b.x, b.y);
        double c = 1.0, s = 0.0, ex = 1.0, ey = 0.0;
        if (bb > 1e-300 && bb > 1e-17 * (fabs(a) + fabs(d))) {
            const double tau = (d - a) / (2.0 * bb);
            const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            ex = b.x / bb;
            ey = b.y / bb;
        }
        sr = make_rot4(c, s, ex, ey);
        rot[blockIdx.x] = sr;
    }
    __syncthreads();
    const double c = sr.x, s = sr.y;
    const double2 e = make_double2(sr.z, sr.w);  // e^{i phi}
    double2* rp = A + (int64_t)p * n;
    double2* rq = A + (int64_t)q * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 ap = rp[j], aq = rq[j];
        const double2 eaq = cmul(e, aq);
        rp[j] = csub(cscale(ap, c), cscale(eaq, s));
        rq[j] = cadd(cscale(ap, s), cscale(eaq, c));
    }
}

// Applies G to columns p and q of A and of the eigenvector accumulator W.
__global__ void jacobi_cols_kernel(double2* __restrict__ A, double2* __restrict__ W, int n, int ne,
                                   int round, const Rot4* __restrict__ rot) {
    int p, q;
    rr_pair(ne, round, blockIdx.x, p, q);
    if (q >= n) return;
    const Rot4 r = rot[blockIdx.x];
    const double c = r.x, s = r.y;
    const double2 ec = make_double2(r.z, -r.w);  // e^{-i phi}
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
        double2* M = i < n ? A : W;
        const int64_t row = (int64_t)(i < n ? i : i - n) * n;
        const double2 ap = M[row + p], aq = M[row + q];
        const double2 eaq = cmul(ec, aq);
        M[row + p] = csub(cscale(ap, c), cscale(eaq, s));
        M[row + q] = cadd(cscale(ap, s), cscale(eaq, c));
    }
}

// sum |A_ij|^2 over i != j and over all (for the stopping test), one block
__global__ void offnorm_kernel(const double2* __restrict__ A, int n, double* __restrict__ out) {
    double off = 0.0, tot = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        const double v = A[e].x * A[e].x + A[e].y * A[e].y;
        tot += v;
        if (e / n != e % n) off += v;
    }
    __shared__ double so[1024], st[1024];
    so[threadIdx.x] = off;
    st[threadIdx.x] = tot;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            so[threadIdx.x] += so[threadIdx.x + w];
            st[threadIdx.x] += st[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = so[0];
        out[1] = st[0];
    }
}

// B <- (B + B^H) / 2
__global__ void hermitise_kernel(double2* __restrict__ B, int n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    if (j < i) return;
    const double2 a = B[(int64_t)i * n + j], b = B[(int64_t)j * n + i];
    const double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    B[(int64_t)i * n + j] = m;
    B[(int64_t)j * n + i] = cconj(m);
}

__global__ void eye_kernel(double2* __restrict__ W, int n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    W[e] = make_double2((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
}

// A final factor in the context precision: F (N x ldu, pad column zero) from the FP64
// N x r matrix Fq.
template <typename R>
__global__ void emit_factors_kernel(const double2* __restrict__ Fq, int64_t N, int r, int ldu,
                                    cplx_t<R>* __restrict__ F) {
    const int64_t tot = N * ldu;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldu;
        const int j = (int)(e % ldu);
        const double2 v = j < r ? Fq[i * r + j] : make_double2(0, 0);
        F[e] = mk((R)v.x, (R)v.y);
    }
}

template <typename R> __global__ void to_real_kernel(const double* __restrict__ s, R* __restrict__ o, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) o[j] = (R)s[j];
}

// ---------------------------------------------------------------- host helpers -------

struct Ws {
    DevBuf work;
    cudaStream_t s;
};

template <typename TA, typename TB, typename Racc, bool HA, bool HB>
void gemm(Ws& w, int M, int Nn, int K, const TA* A, int64_t lda, const TB* B, int64_t ldb,
          double2* C, int64_t ldc, double2 alpha, double2 beta) {
    if (M <= 0 || Nn <= 0) return;
    const int gm = (M + GBM - 1) / GBM, gn = (Nn + GBN - 1) / GBN;
    // split the reduction when the output has too few tiles to fill the GPU
    int ks = 1;
    const int tiles = gm * gn;
    if (tiles < 2 * 152 && K > 4 * GBK) ks = std::min((2 * 152 + tiles - 1) / tiles, K / (4 * GBK));
    ks = std::max(1, std::min(ks, 256));
    int kchunk = (K + ks - 1) / ks;
    kchunk = ((kchunk + GBK - 1) / GBK) * GBK;
    ks = (K + kchunk - 1) / kchunk;
    dim3 grid(gn, gm, ks);
    if (ks == 1) {
        gemm_kernel<TA, TB, Racc, HA, HB><<<grid, GTH, 0, w.s>>>(M, Nn, K, A, lda, B, ldb, C, ldc,
                                                                  alpha, beta, kchunk, nullptr);
        check_launch("gemm_kernel");
    } else {
        w.work.ensure((size_t)ks * M * Nn * sizeof(double2));
        gemm_kernel<TA, TB, Racc, HA, HB><<<grid, GTH, 0, w.s>>>(
            M, Nn, K, A, lda, B, ldb, C, ldc, alpha, beta, kchunk, w.work.as<double2>());
        check_launch("gemm_kernel(split)");
        const int64_t tot = (int64_t)M * Nn;
        splitk_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, w.s>>>(
            M, Nn, ks, w.work.as<double2>(), C, ldc, alpha, beta);
        check_launch("splitk_reduce_kernel");
    }
}

const double2 kOne = {1.0, 0.0}, kZero = {0.0, 0.0}, kMinus = {-1.0, 0.0};

// Y (N x l, FP64, ld l) <- orthonormal basis of its column span, in place: block CGS2 over
// panels of 64 columns, each panel finished by two Cholesky-QR passes.
void orthonormalise(Ws& w, double2* Y, int64_t N, int l, DevBuf& H, DevBuf& P2, DevBuf& Gb,
                    DevBuf& Mb) {
    const int b = 64;
    H.ensure((size_t)l * b * sizeof(double2));
    P2.ensure((size_t)N * b * sizeof(double2));
    Gb.ensure((size_t)b * b * sizeof(double2));
    Mb.ensure((size_t)b * b * sizeof(double2));
    for (int c0 = 0; c0 < l; c0 += b) {
        const int pb = std::min(b, l - c0);
        double2* P = Y + c0;  // panel columns, ld l
        for (int pass = 0; pass < 2 && c0 > 0; ++pass) {
            // H = Q^H P ; P -= Q H   (Q = Y[:, :c0])
            gemm<double2, double2, double, true, false>(w, c0, pb, (int)N, Y, l, P, l, H.as<double2>(),
                                                         pb, kOne, kZero);
            gemm<double2, double2, double, false, false>(w, (int)N, pb, c0, Y, l, H.as<double2>(), pb,
                                                          P, l, kMinus, kOne);
        }
        for (int pass = 0; pass < 2; ++pass) {
            gemm<double2, double2, double, true, false>(w, pb, pb, (int)N, P, l, P, l, Gb.as<double2>(),
                                                         pb, kOne, kZero);
            chol_inv_kernel<<<1, 64, 0, w.s>>>(Gb.as<double2>(), pb, Mb.as<double2>());
            check_launch("chol_inv_kernel");
            // P2 = P M, then copy back into the panel
            gemm<double2, double2, double, false, false>(w, (int)N, pb, pb, P, l, Mb.as<double2>(), pb,
                                                          P2.as<double2>(), pb, kOne, kZero);
            TDAGW_CUDA(cudaMemcpy2DAsync(P, l * sizeof(double2), P2.p, pb * sizeof(double2),
                                         pb * sizeof(double2), N, cudaMemcpyDeviceToDevice, w.s));
        }
    }
}

// Y = K^off X for X (N x l, FP64): the product with K in the context precision; K^off is K
// minus its strict diagonal, or minus its k = k' blocks (kblkF holds them) in k-block mode.
template <typename R>
void apply_koff(Ws& w, const Ctx& c, const double2* X, double2* Y, int l) {
    const int64_t N = c.hm.N;
    gemm<cplx_t<R>, double2, R, false, false>(w, (int)N, l, (int)N, c.K.as<cplx_t<R>>(), N, X, l, Y,
                                              l, kOne, kZero);
    if (c.kdiag) {
        sub_kblock_kernel<R><<<152 * 8, 256, 0, w.s>>>(Y, X, N, l, c.kblkF.as<cplx_t<R>>(), c.hm.Nb * c.hm.Nb);
        check_launch("sub_kblock_kernel");
    } else {
        sub_diag_kernel<R><<<152 * 8, 256, 0, w.s>>>(Y, X, N, l, c.diagK.as<cplx_t<R>>());
        check_launch("sub_diag_kernel");
    }
}

// Hermitian eigen-decomposition of B (n x n, FP64, overwritten by its diagonal form),
// eigenvectors into W; returns the sweeps used.
int jacobi_eigh(Ws& w, double2* B, double2* W, int n) {
    const int ne = n + (n & 1);
    DevBuf rot, nrm;
    rot.ensure((size_t)(ne / 2) * sizeof(Rot4));
    nrm.ensure(2 * sizeof(double));
    eye_kernel<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, w.s>>>(W, n);
    check_launch("eye_kernel");
    int sweep = 0;
    for (; sweep < 60; ++sweep) {
        double h[2];
        offnorm_kernel<<<1, 1024, 0, w.s>>>(B, n, nrm.as<double>());
        TDAGW_CUDA(cudaMemcpyAsync(h, nrm.p, sizeof(h), cudaMemcpyDeviceToHost, w.s));
        TDAGW_CUDA(cudaStreamSynchronize(w.s));
        if (!(h[0] > 1e-26 * h[1]) || h[1] == 0.0) break;
        for (int r = 0; r < ne - 1; ++r) {
            jacobi_rows_kernel<<<ne / 2, 256, 0, w.s>>>(B, n, ne, r, rot.as<Rot4>());
            jacobi_cols_kernel<<<ne / 2, 256, 0, w.s>>>(B, W, n, ne, r, rot.as<Rot4>());
        }
        check_launch("jacobi kernels");
    }
    return sweep;
}

}  // namespace

template <typename R>
void rsvd_compress(Ctx& c, int rank, int oversample, int power_iters, uint64_t seed) {
    Ws w;
    w.s = c.stream;
    const int64_t N = c.hm.N;
    const int l = rank + oversample;
    DevBuf Q, Z, H, P2, Gb, Mb, Bm, Wm;
    Q.ensure((size_t)N * l * sizeof(double2));
    Z.ensure((size_t)N * l * sizeof(double2));
    gauss_kernel<<<152 * 8, 256, 0, w.s>>>(Z.as<double2>(), N * l, seed);
    check_launch("gauss_kernel");
    apply_koff<R>(w, c, Z.as<double2>(), Q.as<double2>(), l);
    orthonormalise(w, Q.as<double2>(), N, l, H, P2, Gb, Mb);
    for (int it = 0; it < 2 * power_iters; ++it) {
        apply_koff<R>(w, c, Q.as<double2>(), Z.as<double2>(), l);
        std::swap(Q.p, Z.p);
        std::swap(Q.bytes, Z.bytes);
        orthonormalise(w, Q.as<double2>(), N, l, H, P2, Gb, Mb);
    }
    // Z = K^off Q = B^H (B = Q^H K^off), core B B^H = Z^H Z
    apply_koff<R>(w, c, Q.as<double2>(), Z.as<double2>(), l);
    Bm.ensure((size_t)l * l * sizeof(double2));
    Wm.ensure((size_t)l * l * sizeof(double2));
    gemm<double2, double2, double, true, false>(w, l, l, (int)N, Z.as<double2>(), l, Z.as<double2>(),
                                                 l, Bm.as<double2>(), l, kOne, kZero);
    hermitise_kernel<<<(unsigned)(((int64_t)l * l + 255) / 256), 256, 0, w.s>>>(Bm.as<double2>(), l);
    check_launch("hermitise_kernel");
    jacobi_eigh(w, Bm.as<double2>(), Wm.as<double2>(), l);
    // eigenvalues sigma^2, largest first
    std::vector<double2> hb((size_t)l * l);
    TDAGW_CUDA(cudaMemcpyAsync(hb.data(), Bm.p, hb.size() * sizeof(double2), cudaMemcpyDeviceToHost, w.s));
    std::vector<double2> hw((size_t)l * l);
    TDAGW_CUDA(cudaMemcpyAsync(hw.data(), Wm.p, hw.size() * sizeof(double2), cudaMemcpyDeviceToHost, w.s));
    TDAGW_CUDA(cudaStreamSynchronize(w.s));
    std::vector<double> lam(l);
    for (int i = 0; i < l; ++i) lam[i] = hb[(size_t)i * l + i].x;
    std::vector<int> idx(l);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    const double s0 = std::sqrt(std::max(0.0, lam[idx[0]]));
    std::vector<double2> wr((size_t)l * rank), wv((size_t)l * rank);
    std::vector<double> sv(rank);
    for (int j = 0; j < rank; ++j) {
        const int src = idx[j];
        double sj = std::sqrt(std::max(0.0, lam[src]));
        if (!(sj > 1e-7 * s0)) sj = 0.0;
        sv[j] = sj;
        for (int i = 0; i < l; ++i) {
            const double2 e = hw[(size_t)i * l + src];
            wr[(size_t)i * rank + j] = e;
            wv[(size_t)i * rank + j] = sj > 0.0 ? make_double2(e.x / sj, e.y / sj) : make_double2(0.0, 0.0);
        }
    }
    // U = Q W_r and V = Z W_r diag(1 / sigma), FP64
    DevBuf Wr, Uq, Vq, dS;
    Wr.ensure(wr.size() * sizeof(double2));
    Uq.ensure((size_t)N * rank * sizeof(double2));
    Vq.ensure((size_t)N * rank * sizeof(double2));
    TDAGW_CUDA(cudaMemcpyAsync(Wr.p, wr.data(), wr.size() * sizeof(double2), cudaMemcpyHostToDevice, w.s));
    gemm<double2, double2, double, false, false>(w, (int)N, rank, l, Q.as<double2>(), l, Wr.as<double2>(),
                                                 rank, Uq.as<double2>(), rank, kOne, kZero);
    TDAGW_CUDA(cudaStreamSynchronize(w.s));
    TDAGW_CUDA(cudaMemcpyAsync(Wr.p, wv.data(), wv.size() * sizeof(double2), cudaMemcpyHostToDevice, w.s));
    gemm<double2, double2, double, false, false>(w, (int)N, rank, l, Z.as<double2>(), l, Wr.as<double2>(),
                                                 rank, Vq.as<double2>(), rank, kOne, kZero);
    dS.ensure(rank * sizeof(double));
    TDAGW_CUDA(cudaMemcpyAsync(dS.p, sv.data(), rank * sizeof(double), cudaMemcpyHostToDevice, w.s));
    TDAGW_CUDA(cudaStreamSynchronize(w.s));
    // release the sketch workspace before allocating the factors
    Q.release();
    Z.release();
    P2.release();
    w.work.release();
    using C = cplx_t<R>;
    const int ldu = rank + (rank & 1);
    c.U.ensure((size_t)N * ldu * sizeof(C));
    c.V.ensure((size_t)N * ldu * sizeof(C));
    emit_factors_kernel<R><<<152 * 8, 256, 0, w.s>>>(Uq.as<double2>(), N, rank, ldu, c.U.as<C>());
    check_launch("emit_factors_kernel");
    emit_factors_kernel<R><<<152 * 8, 256, 0, w.s>>>(Vq.as<double2>(), N, rank, ldu, c.V.as<C>());
    check_launch("emit_factors_kernel");
    c.S.ensure(rank * sizeof(R));
    to_real_kernel<R><<<(rank + 255) / 256, 256, 0, w.s>>>(dS.as<double>(), c.S.as<R>(), rank);
    check_launch("to_real_kernel");
    c.diagF.ensure(N * sizeof(C));
    TDAGW_CUDA(cudaMemcpyAsync(c.diagF.p, c.diagK.p, N * sizeof(C), cudaMemcpyDeviceToDevice, w.s));
    c.rank = rank;
    c.ysplit = choose_ysplit(rank, N);
    c.ypart.ensure((size_t)c.ysplit * rank * sizeof(C));
    c.ytil.ensure((size_t)ldu * sizeof(C));
    TDAGW_CUDA(cudaMemsetAsync(c.ytil.p, 0, ldu * sizeof(C), w.s));
    TDAGW_CUDA(cudaStreamSynchronize(w.s));
}

template void rsvd_compress<float>(Ctx&, int, int, int, uint64_t);
template void rsvd_compress<double>(Ctx&, int, int, int, uint64_t);

// Channel-wise factors (Eq. svd-channel-wise).  Every off-diagonal channel A = K^pq (p < q,
// Nk x Nk, gathered contiguously in the context precision) gets a randomised truncated SVD
// by the same range finder as above, now for a general (non-Hermitian) matrix:
//   Q = orth(A Omega); repeat power_iters times: Q = orth(A orth(A^H Q))
//   Z = A^H Q = B^H (B = Q^H A, l x Nk);  B B^H = Z^H Z = W diag(lambda) W^H (Jacobi)
//   sigma_j = sqrt(lambda_j),  U = Q W_r,  V = Z W_r diag(1 / sigma)   (B = W Sigma V^H)
// The core squares the singular values, so sigma_j below 1e-7 sigma_0 is not resolved in
// FP64 and is dropped together with those below rel_tol sigma_0 (a vanishing channel keeps
// nothing).  Channel q -> p is (K^pq)^H = V^pq S^pq (U^pq)^H.
template <typename R>
void rsvd_channels(Ctx& c, int rank, int oversample, int power_iters, uint64_t seed, double rel_tol) {
    using C = cplx_t<R>;
    Ws w;
    w.s = c.stream;
    const HostModel& h = c.hm;
    const int P = h.Nb * h.Nb, Nk = h.Nk;
    const int l = std::max(1, std::min(rank + oversample, Nk));
    const double floor_rel = std::max(rel_tol, 1e-7);
    struct Fac {
        DevBuf U, V;
        std::vector<double> S;
    };
    std::vector<Fac> fac(P * P);
    std::vector<int> z(P * P, 0);
    DevBuf A, Q, Z, H, P2, Gb, Mb, Bm, Wm, Wr;
    if (rank > 0) {
        A.ensure((size_t)Nk * Nk * sizeof(C));
        Q.ensure((size_t)Nk * l * sizeof(double2));
        Z.ensure((size_t)Nk * l * sizeof(double2));
        Bm.ensure((size_t)l * l * sizeof(double2));
        Wm.ensure((size_t)l * l * sizeof(double2));
    }
    std::vector<double2> hb((size_t)l * l), hw((size_t)l * l);
    for (int p = 0; p < P && rank > 0; ++p)
        for (int q = p + 1; q < P; ++q) {
            launch_ch_gather<R>(c, p, q, A.p, Nk, w.s);
            const C* Ap = A.as<C>();
            gauss_kernel<<<152 * 8, 256, 0, w.s>>>(Z.as<double2>(), (int64_t)Nk * l,
                                                   seed ^ splitmix64_host((uint64_t)(p * P + q) + 1));
            check_launch("gauss_kernel");
            gemm<C, double2, R, false, false>(w, Nk, l, Nk, Ap, Nk, Z.as<double2>(), l, Q.as<double2>(), l,
                                              kOne, kZero);
            orthonormalise(w, Q.as<double2>(), Nk, l, H, P2, Gb, Mb);
            for (int it = 0; it < power_iters; ++it) {
                gemm<C, double2, R, true, false>(w, Nk, l, Nk, Ap, Nk, Q.as<double2>(), l, Z.as<double2>(), l,
                                                 kOne, kZero);
                orthonormalise(w, Z.as<double2>(), Nk, l, H, P2, Gb, Mb);
                gemm<C, double2, R, false, false>(w, Nk, l, Nk, Ap, Nk, Z.as<double2>(), l, Q.as<double2>(),
                                                  l, kOne, kZero);
                orthonormalise(w, Q.as<double2>(), Nk, l, H, P2, Gb, Mb);
            }
            gemm<C, double2, R, true, false>(w, Nk, l, Nk, Ap, Nk, Q.as<double2>(), l, Z.as<double2>(), l,
                                             kOne, kZero);
            gemm<double2, double2, double, true, false>(w, l, l, Nk, Z.as<double2>(), l, Z.as<double2>(), l,
                                                        Bm.as<double2>(), l, kOne, kZero);
            hermitise_kernel<<<(unsigned)(((int64_t)l * l + 255) / 256), 256, 0, w.s>>>(Bm.as<double2>(), l);
            check_launch("hermitise_kernel");
            jacobi_eigh(w, Bm.as<double2>(), Wm.as<double2>(), l);
            TDAGW_CUDA(cudaMemcpyAsync(hb.data(), Bm.p, hb.size() * sizeof(double2), cudaMemcpyDeviceToHost, w.s));
            TDAGW_CUDA(cudaMemcpyAsync(hw.data(), Wm.p, hw.size() * sizeof(double2), cudaMemcpyDeviceToHost, w.s));
            TDAGW_CUDA(cudaStreamSynchronize(w.s));
            std::vector<int> idx(l);
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(),
                             [&](int a, int b) { return hb[(size_t)a * l + a].x > hb[(size_t)b * l + b].x; });
            const double s0 = std::sqrt(std::max(0.0, hb[(size_t)idx[0] * l + idx[0]].x));
            std::vector<double> sv;
            for (int j = 0; j < std::min(rank, l); ++j) {
                const double sj = std::sqrt(std::max(0.0, hb[(size_t)idx[j] * l + idx[j]].x));
                if (!(sj > 0.0) || sj <= floor_rel * s0) break;
                sv.push_back(sj);
            }
            const int zz = (int)sv.size();
            z[p * P + q] = z[q * P + p] = zz;
            if (zz == 0) continue;
            // U = Q W_r and V = Z W_r diag(1 / sigma), FP64
            std::vector<double2> wr((size_t)l * zz), wv((size_t)l * zz);
            for (int j = 0; j < zz; ++j)
                for (int i = 0; i < l; ++i) {
                    const double2 e = hw[(size_t)i * l + idx[j]];
                    wr[(size_t)i * zz + j] = e;
                    wv[(size_t)i * zz + j] = make_double2(e.x / sv[j], e.y / sv[j]);
                }
            Fac& fc = fac[p * P + q];
            fc.S = sv;
            fc.U.ensure((size_t)Nk * zz * sizeof(double2));
            fc.V.ensure((size_t)Nk * zz * sizeof(double2));
            Wr.ensure((size_t)l * zz * sizeof(double2));
            TDAGW_CUDA(cudaMemcpyAsync(Wr.p, wr.data(), wr.size() * sizeof(double2), cudaMemcpyHostToDevice, w.s));
            gemm<double2, double2, double, false, false>(w, Nk, zz, l, Q.as<double2>(), l, Wr.as<double2>(), zz,
                                                         fc.U.as<double2>(), zz, kOne, kZero);
            TDAGW_CUDA(cudaStreamSynchronize(w.s));
            TDAGW_CUDA(cudaMemcpyAsync(Wr.p, wv.data(), wv.size() * sizeof(double2), cudaMemcpyHostToDevice, w.s));
            gemm<double2, double2, double, false, false>(w, Nk, zz, l, Z.as<double2>(), l, Wr.as<double2>(), zz,
                                                         fc.V.as<double2>(), zz, kOne, kZero);
            TDAGW_CUDA(cudaStreamSynchronize(w.s));
        }
    A.release();
    Q.release();
    Z.release();
    P2.release();
    w.work.release();
    // segment layout for the final ranks, then every channel into place
    ch_layout(c, z);
    ChannelFactors& f = c.ch;
    const ChMeta& m = f.m;
    std::vector<R> hs((size_t)std::max<long long>(m.stot, 1), (R)0);
    C* Vd = f.V.as<C>();
    C* Ud = f.U.as<C>();
    for (int p = 0; p < P; ++p)
        for (int q = p + 1; q < P; ++q) {
            const int zz = z[p * P + q];
            if (zz == 0) continue;
            const Fac& fc = fac[p * P + q];
            // channel p -> q: U^pq into U segment p, V^pq into V segment q
            launch_ch_place<R>(fc.U.as<double2>(), Nk, zz, Ud + m.ubase[p], m.ldw[p], f.uoff[p * P + q], w.s);
            launch_ch_place<R>(fc.V.as<double2>(), Nk, zz, Vd + m.vbase[q], m.ldv[q], f.voff[q * P + p], w.s);
            // channel q -> p = (K^pq)^H: U^qp = V^pq into U segment q, V^qp = U^pq into V segment p
            launch_ch_place<R>(fc.V.as<double2>(), Nk, zz, Ud + m.ubase[q], m.ldw[q], f.uoff[q * P + p], w.s);
            launch_ch_place<R>(fc.U.as<double2>(), Nk, zz, Vd + m.vbase[p], m.ldv[p], f.voff[p * P + q], w.s);
            for (int j = 0; j < zz; ++j) {
                hs[m.sbase[q] + f.voff[q * P + p] + j] = (R)fc.S[j];
                hs[m.sbase[p] + f.voff[p * P + q] + j] = (R)fc.S[j];
            }
        }
    ch_fill_diag_from_kernel<R>(c);
    TDAGW_CUDA(cudaMemcpyAsync(f.S.p, hs.data(), hs.size() * sizeof(R), cudaMemcpyHostToDevice, w.s));
    TDAGW_CUDA(cudaStreamSynchronize(w.s));
    f.valid = true;
}

template void rsvd_channels<float>(Ctx&, int, int, int, uint64_t, double);
template void rsvd_channels<double>(Ctx&, int, int, int, uint64_t, double);

}  // namespace tdagw
