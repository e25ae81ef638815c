// High-harmonic spectrum of recorded currents (Sec. "SVD acceleration of TD-aGW"):
//   HHG_b(w) = | w sum_{n=0..T_b} J_b(t_n) e^{-i w t_n} dt |^2,   t_n = n dt,
// for B trajectories (an angle or frequency sweep) at nfreq angular frequencies.  One
// thread per (frequency, trajectory); the trajectory's current is staged through shared
// memory in chunks; the phasor e^{-i w t_n} advances by one complex multiplication per step
// and is recomputed exactly at the start of every chunk, so rounding does not accumulate
// over long runs.  FP64 throughout.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace tdagw {

namespace {

constexpr int kHhgThreads = 128, kHhgChunk = 256;

__global__ void __launch_bounds__(kHhgThreads)
hhg_kernel(const double* __restrict__ J, int64_t stride, int B, const int* __restrict__ steps, double dt,
           const double* __restrict__ omega, int nfreq, double* __restrict__ out) {
    __shared__ double js[kHhgChunk];
    const int b = blockIdx.y;
    const int f = blockIdx.x * kHhgThreads + threadIdx.x;
    const int T = steps[b];
    const double w = f < nfreq ? omega[f] : 0.0;
    double sdt, cdt;
    sincos(w * dt, &sdt, &cdt);
    double re = 0.0, im = 0.0;
    for (int n0 = 0; n0 <= T; n0 += kHhgChunk) {
        const int cnt = min(kHhgChunk, T + 1 - n0);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += kHhgThreads) js[e] = J[((int64_t)(n0 + e) * B + b) * stride];
        __syncthreads();
        double s0, c0;
        sincos(w * ((double)n0 * dt), &s0, &c0);
        double cr = c0, ci = -s0;  // e^{-i w t_n}
        for (int e = 0; e < cnt; ++e) {
            re = fma(js[e], cr, re);
            im = fma(js[e], ci, im);
            const double nr = cr * cdt + ci * sdt;  // times e^{-i w dt}
            const double ni = ci * cdt - cr * sdt;
            cr = nr;
            ci = ni;
        }
    }
    if (f < nfreq) {
        const double a = w * dt;
        out[(int64_t)f * B + b] = a * a * (re * re + im * im);
    }
}

}  // namespace

void hhg_spectrum(const double* J, int64_t rows, int64_t stride, int B, const int* steps, double dt,
                  const double* omega, int nfreq, double* out, cudaStream_t s) {
    int tmax = 0;
    for (int b = 0; b < B; ++b) tmax = std::max(tmax, steps[b]);
    TDAGW_REQUIRE(rows >= (int64_t)tmax + 1, TDAGW_ERR_INVALID_ARG, "fewer rows than steps + 1");
    const size_t nJ = ((size_t)rows * B - 1) * stride + 1;  // last element read: ((rows - 1) B + B - 1) stride
    DevBuf dJ, dS, dW, dO;
    dJ.ensure(nJ * sizeof(double));
    dS.ensure((size_t)B * sizeof(int));
    dW.ensure((size_t)nfreq * sizeof(double));
    dO.ensure((size_t)nfreq * B * sizeof(double));
    TDAGW_CUDA(cudaMemcpyAsync(dJ.p, J, nJ * sizeof(double), cudaMemcpyHostToDevice, s));
    TDAGW_CUDA(cudaMemcpyAsync(dS.p, steps, (size_t)B * sizeof(int), cudaMemcpyHostToDevice, s));
    TDAGW_CUDA(cudaMemcpyAsync(dW.p, omega, (size_t)nfreq * sizeof(double), cudaMemcpyHostToDevice, s));
    dim3 grid((unsigned)((nfreq + kHhgThreads - 1) / kHhgThreads), (unsigned)B);
    hhg_kernel<<<grid, kHhgThreads, 0, s>>>(dJ.as<double>(), stride, B, dS.as<int>(), dt, dW.as<double>(), nfreq,
                                            dO.as<double>());
    check_launch("hhg_kernel");
    TDAGW_CUDA(cudaMemcpyAsync(out, dO.p, (size_t)nfreq * B * sizeof(double), cudaMemcpyDeviceToHost, s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
}

}  // namespace tdagw
