// Device construction of the dense kernel (Eq. bse-direct-def for the lattice model, plus the
// optional exchange term of Eq. bse-exchange-def),
// sampled reads of it, precision conversions at the boundary, and the pulse sample table.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace tdagw {

namespace {

constexpr int kBuildThreads = 128;

// One thread per (k, k') pair of grid points: it forms the Nb x Nb overlap
// O = U_k^+ U_k' in FP64 and writes the Nb^2 x Nb^2 block
//   K[(k n m), (k' n' m')] = -W(k - k') O[n][n'] conj(O[m][m'])
// row by row; consecutive threads hold consecutive k', so each row segment of the block
// (Nb^2 complex) is adjacent to its neighbour's and the stores coalesce.
// With the exchange term (Mx != nullptr) every entry also gets
//   sum_g vG[g] Mx[k][g][n m] conj(Mx[k'][g][n' m'])   (Eq. bse-exchange-def, eight G).
template <typename R, int NB>
__global__ void __launch_bounds__(kBuildThreads)
build_kernel_kernel(const double2* __restrict__ U, const double* __restrict__ Wtab, int L,
                    int Nk, const double2* __restrict__ Mx, const double* __restrict__ vG,
                    cplx_t<R>* __restrict__ K) {
    using C = cplx_t<R>;
    constexpr int NB2 = NB * NB;
    __shared__ double2 Uk[NB * NB];
    __shared__ double2 Mk[8 * NB2];
    const int k = blockIdx.y;
    const int kp = blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x < NB * NB) Uk[threadIdx.x] = U[(size_t)k * NB * NB + threadIdx.x];
    if (Mx)
        for (int e = threadIdx.x; e < 8 * NB2; e += blockDim.x) Mk[e] = Mx[(size_t)k * 8 * NB2 + e];
    __syncthreads();
    if (kp >= Nk) return;
    double2 Ukp[NB * NB];
#pragma unroll
    for (int i = 0; i < NB * NB; ++i) Ukp[i] = U[(size_t)kp * NB * NB + i];
    // U layout: [k][orbital][band]
    double2 O[NB][NB];
#pragma unroll
    for (int n = 0; n < NB; ++n)
#pragma unroll
        for (int np = 0; np < NB; ++np) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int o = 0; o < NB; ++o) s = cfmac(Uk[o * NB + n], Ukp[o * NB + np], s);
            O[n][np] = s;
        }
    int di = (k / L) - (kp / L), dj = (k % L) - (kp % L);
    di += di < 0 ? L : 0;
    dj += dj < 0 ? L : 0;
    const double w = -Wtab[di * L + dj];
    const int64_t N = (int64_t)Nk * NB2;
#pragma unroll
    for (int n = 0; n < NB; ++n)
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            C* row = K + ((int64_t)k * NB2 + n * NB + m) * N + (int64_t)kp * NB2;
#pragma unroll
            for (int np = 0; np < NB; ++np)
#pragma unroll
                for (int mp = 0; mp < NB; ++mp) {
                    double2 v = cscale(cmulc(O[n][np], O[m][mp]), w);
                    if (Mx) {
                        const double2* Mkp = Mx + (size_t)kp * 8 * NB2 + np * NB + mp;
                        for (int g = 0; g < 8; ++g)
                            v = cadd(v, cscale(cmulc(Mk[g * NB2 + n * NB + m], Mkp[g * NB2]), vG[g]));
                    }
                    row[np * NB + mp] = mk((R)v.x, (R)v.y);
                }
        }
}

template <typename R>
__global__ void gather_kernel(const cplx_t<R>* __restrict__ K, int64_t N,
                              const int64_t* __restrict__ rows, const int64_t* __restrict__ cols,
                              int64_t n, double2* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cplx_t<R> v = K[rows[i] * N + cols[i]];
    out[i] = make_double2((double)v.x, (double)v.y);
}

template <typename R>
__global__ void convert_in_kernel(const double2* __restrict__ src, cplx_t<R>* __restrict__ dst,
                                  int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = mk((R)src[i].x, (R)src[i].y);
}

template <typename R>
__global__ void convert_out_kernel(const cplx_t<R>* __restrict__ src, double2* __restrict__ dst,
                                   int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}

// E(t_start + j dt / 2) for j < nsamp: every RK4 stage time of the run (Algorithm: the
// stage times of classical RK4 are t_n, t_n + dt/2 (twice) and t_n + dt).
__device__ double field_value(int kind, double E0, double omega, double t0, double sigma, double Tp,
                              double t) {
    double e = 0.0;
    if (kind == TDAGW_FIELD_GAUSS_COS) {
        const double u = t - t0;
        e = E0 * exp(-(u * u) / (2.0 * sigma * sigma)) * cos(omega * t);
    } else if (kind == TDAGW_FIELD_CONST) {
        e = E0;
    } else if (kind == TDAGW_FIELD_SIN2_SIN) {
        if (t >= 0.0 && t <= Tp) {
            const double s = sin(3.14159265358979323846 * t / Tp);
            e = E0 * s * s * sin(omega * t);
        }
    }
    return e;
}

__global__ void field_table_kernel(int kind, double E0, double omega, double t0, double sigma,
                                   double Tp, double t_start, double dt, int64_t nsamp,
                                   double* __restrict__ out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nsamp) return;
    out[j] = field_value(kind, E0, omega, t0, sigma, Tp, t_start + 0.5 * dt * (double)j);
}

// all analytic tables of a batch in one launch: row q of out (stride ldE) holds the
// half-step samples of trajectory q (table-kind rows are left to the caller)
__global__ void field_tables_kernel(const FieldParams* __restrict__ p, int B, int64_t ldE, double dt,
                                    double* __restrict__ out) {
    for (int q = blockIdx.y; q < B; q += gridDim.y) {
        const FieldParams f = p[q];
        if (f.kind == TDAGW_FIELD_TABLE) continue;
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < f.nsamp;
             j += (int64_t)gridDim.x * blockDim.x)
            out[(int64_t)q * ldE + j] = field_value(f.kind, f.E0, f.omega, f.t0, f.sigma, f.Tp, 0.5 * dt * (double)j);
    }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 32) {
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

template <typename R>
void launch_build_kernel(const Ctx& c, cudaStream_t s) {
    const HostModel& hm = c.hm;
    dim3 grid((hm.Nk + kBuildThreads - 1) / kBuildThreads, hm.Nk);
    auto* K = c.K.as<cplx_t<R>>();
    const double2* Mx = hm.Mx.empty() ? nullptr : c.Mxd.as<double2>();
    const double* vG = hm.Mx.empty() ? nullptr : c.vGd.as<double>();
    if (hm.Nb == 2)
        build_kernel_kernel<R, 2><<<grid, kBuildThreads, 0, s>>>(c.Ud.as<double2>(), c.Wd.as<double>(), hm.L,
                                                                 hm.Nk, Mx, vG, K);
    else
        build_kernel_kernel<R, 4><<<grid, kBuildThreads, 0, s>>>(c.Ud.as<double2>(), c.Wd.as<double>(), hm.L,
                                                                 hm.Nk, Mx, vG, K);
    check_launch("build_kernel_kernel");
}

template <typename R>
void launch_gather_entries(const Ctx& c, const int64_t* rows, const int64_t* cols, int64_t n,
                           double2* out, cudaStream_t s) {
    if (n <= 0) return;
    gather_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.K.as<cplx_t<R>>(), c.hm.N,
                                                                  rows, cols, n, out);
    check_launch("gather_kernel");
}

template <typename R>
void launch_convert_in(const double2* src, void* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    convert_in_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(src, static_cast<cplx_t<R>*>(dst), n);
    check_launch("convert_in_kernel");
}

template <typename R>
void launch_convert_out(const void* src, double2* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    convert_out_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const cplx_t<R>*>(src),
                                                            dst, n);
    check_launch("convert_out_kernel");
}

void launch_field_table(const tdagw_field& f, double t_start, double dt, int64_t nsamp,
                        double* out, cudaStream_t s) {
    field_table_kernel<<<(unsigned)((nsamp + 255) / 256), 256, 0, s>>>(
        f.kind, f.E0, f.omega, f.t0, f.sigma, f.T_pulse, t_start, dt, nsamp, out);
    check_launch("field_table_kernel");
}

void launch_field_tables(const FieldParams* p_dev, int B, int64_t max_nsamp, int64_t ldE, double dt,
                         double* out, cudaStream_t s) {
    const unsigned gx = (unsigned)std::min<int64_t>(64, (max_nsamp + 255) / 256);
    const unsigned gy = (unsigned)std::min(B, 4096);
    field_tables_kernel<<<dim3(std::max(1u, gx), std::max(1u, gy)), 256, 0, s>>>(p_dev, B, ldE, dt, out);
    check_launch("field_tables_kernel");
}

#define INST(R)                                                                            \
    template void launch_build_kernel<R>(const Ctx&, cudaStream_t);                        \
    template void launch_gather_entries<R>(const Ctx&, const int64_t*, const int64_t*,     \
                                           int64_t, double2*, cudaStream_t);               \
    template void launch_convert_in<R>(const double2*, void*, int64_t, cudaStream_t);      \
    template void launch_convert_out<R>(const void*, double2*, int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace tdagw
