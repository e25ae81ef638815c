// Channel-wise compressed kernel (Sec. "SVD analysis of electron-hole kernel", Eq.
// svd-channel-wise): storage layout, host exchange of the factors, and the stage-wise
// apply
//
//   dSigma[k P + p] = sum_k' K^pp[k, k'] x[k' P + p] + sum_{q != p} U^pq (S^pq o ((V^pq)^H x_q))
//
// as two passes.  V pass: for every input pair q one matrix-vector product of the V
// segment q (Nk rows; row k' holds V^pq[k', :] of all channels into q) with x_q, giving all
// (V^pq)^H x_q at once, scaled by S.  U pass: for every output pair p one product of the U
// segment p (row k holds U^pq[k, :] of all channels out of p, then the dense row K^pp[k, :])
// with the vector [S o y of those channels ; x_p].
#include <algorithm>

#include "common.cuh"

namespace tdagw {

namespace {

template <typename R>
__global__ void ch_gather_kernel(const cplx_t<R>* __restrict__ K, int64_t N, int P, int Nk, int p,
                                 int q, cplx_t<R>* __restrict__ dst, int64_t ld) {
    const int64_t n = (int64_t)Nk * Nk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / Nk, kp = e % Nk;
        dst[k * ld + kp] = K[(k * P + p) * N + kp * P + q];
    }
}

template <typename R>
__global__ void ch_place_kernel(const double2* __restrict__ src, int Nk, int z, cplx_t<R>* __restrict__ dst,
                                int64_t ld, int off) {
    const int64_t n = (int64_t)Nk * z;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / z, j = e % z;
        dst[k * ld + off + j] = mk((R)src[e].x, (R)src[e].y);
    }
}

// V pass: part[b][col] = sum over the k' of split b of conj(V_q[k'][c]) x[k' P + q] for
// every column col = sbase[q] + c of every segment (one thread per column).
template <typename R>
__global__ void __launch_bounds__(256)
ch_vpass_kernel(ChMeta m, const cplx_t<R>* __restrict__ V, const cplx_t<R>* __restrict__ x,
                cplx_t<R>* __restrict__ part, int nsplit) {
    using C = cplx_t<R>;
    const int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (col >= m.stot) return;
    int q = 0;
    while (q + 1 < m.P && m.sbase[q + 1] <= col) ++q;
    const int c = (int)(col - m.sbase[q]);
    const int ld = m.ldv[q];
    const int k0 = (int)((int64_t)blockIdx.y * m.Nk / nsplit), k1 = (int)((int64_t)(blockIdx.y + 1) * m.Nk / nsplit);
    C acc = mk((R)0, (R)0);
    const C* v = V + m.vbase[q] + c;
    for (int k = k0; k < k1; ++k) acc = cfmac(v[(int64_t)k * ld], __ldg(x + (int64_t)k * m.P + q), acc);
    part[(int64_t)blockIdx.y * m.stot + col] = acc;
}

// U pass: one warp per output row (p, k) of the U segments.
template <typename R>
__global__ void __launch_bounds__(256)
ch_upass_kernel(ChMeta m, const cplx_t<R>* __restrict__ U, const cplx_t<R>* __restrict__ ytil,
                const int* __restrict__ gidx, const cplx_t<R>* __restrict__ x, cplx_t<R>* __restrict__ y) {
    using C = cplx_t<R>;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)m.P * m.Nk) return;
    const int p = (int)(w / m.Nk), k = (int)(w % m.Nk);
    const int nl = m.nlr[p];
    const C* row = U + m.ubase[p] + (int64_t)k * m.ldw[p];
    const int* g = gidx + m.gbase[p];
    C acc = mk((R)0, (R)0);
    for (int c = lane; c < nl; c += 32) acc = cfma(row[c], ytil[g[c]], acc);
    for (int c = lane; c < m.Nk; c += 32) acc = cfma(row[nl + c], x[(int64_t)c * m.P + p], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) y[(int64_t)k * m.P + p] = acc;
}

int vpass_splits(const ChMeta& m) {
    const int64_t want = (4 * 152 * 256) / std::max<int64_t>(m.stot, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, 4096), std::max(1, m.Nk / 4)));
}

}  // namespace

void ch_layout(Ctx& c, const std::vector<int>& z) {
    const HostModel& h = c.hm;
    const int P = h.Nb * h.Nb, Nk = h.Nk;
    ChannelFactors& f = c.ch;
    f.valid = false;
    f.tc_valid = false;
    f.z = z;
    f.zmax = 0;
    for (int p = 0; p < P; ++p) f.z[p * P + p] = 0;
    for (int e = 0; e < P * P; ++e) f.zmax = std::max(f.zmax, f.z[e]);
    f.voff.assign(P * P, 0);
    f.uoff.assign(P * P, 0);
    ChMeta& m = f.m;
    m = ChMeta{};
    m.P = P;
    m.Nk = Nk;
    for (int q = 0; q < P; ++q) {
        int o = 0;
        for (int p = 0; p < P; ++p) {
            if (p == q) continue;
            f.voff[q * P + p] = o;
            o += f.z[p * P + q];
        }
        m.ldv[q] = o + (o & 1);
    }
    for (int p = 0; p < P; ++p) {
        int o = 0;
        for (int q = 0; q < P; ++q) {
            if (q == p) continue;
            f.uoff[p * P + q] = o;
            o += f.z[p * P + q];
        }
        m.nlr[p] = o;
        const int w = o + Nk;
        m.ldw[p] = w + (w & 1);
    }
    long long vb = 0, ub = 0, sb = 0, gb = 0;
    for (int q = 0; q < P; ++q) {
        m.vbase[q] = vb;
        m.ubase[q] = ub;
        m.sbase[q] = sb;
        m.gbase[q] = gb;
        vb += (long long)Nk * m.ldv[q];
        ub += (long long)Nk * m.ldw[q];
        sb += m.ldv[q];
        gb += m.nlr[q];
    }
    m.vtot = vb;
    m.utot = ub;
    m.stot = sb;
    m.gtot = gb;
    f.gidx_host.assign((size_t)std::max<long long>(gb, 1), 0);
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q) {
            if (q == p) continue;
            for (int j = 0; j < f.z[p * P + q]; ++j)
                f.gidx_host[m.gbase[p] + f.uoff[p * P + q] + j] =
                    (int)(m.sbase[q] + f.voff[q * P + p] + j);
        }
    cudaStream_t s = c.stream;
    const size_t csz = c.csz, rsz = csz / 2;
    f.V.ensure((size_t)std::max<long long>(vb, 1) * csz);
    f.U.ensure((size_t)ub * csz);
    f.S.ensure((size_t)std::max<long long>(sb, 1) * rsz);
    f.Y.ensure((size_t)std::max<long long>(sb, 1) * csz);
    f.gidx.ensure(f.gidx_host.size() * sizeof(int));
    // partials of the stage-wise V pass, allocated here: the stage-wise apply may run
    // inside a CUDA graph capture, where no allocation is allowed
    f.part.ensure((size_t)vpass_splits(m) * std::max<long long>(sb, 1) * csz);
    TDAGW_CUDA(cudaMemsetAsync(f.V.p, 0, f.V.bytes, s));
    TDAGW_CUDA(cudaMemsetAsync(f.U.p, 0, f.U.bytes, s));
    TDAGW_CUDA(cudaMemsetAsync(f.S.p, 0, f.S.bytes, s));
    TDAGW_CUDA(cudaMemsetAsync(f.Y.p, 0, f.Y.bytes, s));
    TDAGW_CUDA(cudaMemcpyAsync(f.gidx.p, f.gidx_host.data(), f.gidx_host.size() * sizeof(int),
                               cudaMemcpyHostToDevice, s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
}

template <typename R>
void launch_ch_gather(const Ctx& c, int p, int q, void* dst, int64_t ld, cudaStream_t s) {
    const HostModel& h = c.hm;
    ch_gather_kernel<R><<<152 * 4, 256, 0, s>>>(c.K.as<cplx_t<R>>(), h.N, h.Nb * h.Nb, h.Nk, p, q,
                                                static_cast<cplx_t<R>*>(dst), ld);
    check_launch("ch_gather_kernel");
}

template <typename R>
void launch_ch_place(const double2* src, int Nk, int z, void* dst, int64_t ld, int off, cudaStream_t s) {
    if (z <= 0) return;
    ch_place_kernel<R><<<152 * 4, 256, 0, s>>>(src, Nk, z, static_cast<cplx_t<R>*>(dst), ld, off);
    check_launch("ch_place_kernel");
}

template <typename R>
void ch_fill_diag_from_kernel(Ctx& c) {
    ChannelFactors& f = c.ch;
    cplx_t<R>* U = f.U.as<cplx_t<R>>();
    for (int p = 0; p < f.m.P; ++p)
        launch_ch_gather<R>(c, p, p, U + f.m.ubase[p] + f.m.nlr[p], f.m.ldw[p], c.stream);
}

template <typename R>
void set_channel_factors(Ctx& c, int rank, const int* ranks, const double* U, const double* S,
                         const double* V, const double* D) {
    const HostModel& h = c.hm;
    const int P = h.Nb * h.Nb, Nk = h.Nk;
    std::vector<int> z(P * P, rank);
    if (ranks)
        for (int e = 0; e < P * P; ++e) z[e] = ranks[e];
    for (int p = 0; p < P; ++p) z[p * P + p] = 0;
    for (int e = 0; e < P * P; ++e)
        TDAGW_REQUIRE(z[e] >= 0 && z[e] <= rank, TDAGW_ERR_INVALID_ARG, "channel rank out of range");
    ch_layout(c, z);
    ChannelFactors& f = c.ch;
    const ChMeta& m = f.m;
    cudaStream_t s = c.stream;
    // the factors, packed into the segment layout in FP64 on the host
    std::vector<double2> hv((size_t)m.vtot, make_double2(0, 0)), hu((size_t)m.utot, make_double2(0, 0));
    std::vector<R> hs((size_t)std::max<long long>(m.stot, 1), (R)0);
    auto at = [&](const double* a, int p, int q, int k, int j) {
        const size_t e = (((size_t)(p * P + q) * Nk + k) * rank + j) * 2;
        return make_double2(a[e], a[e + 1]);
    };
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q) {
            const int zz = z[p * P + q];
            if (p == q || zz == 0) continue;
            for (int k = 0; k < Nk; ++k)
                for (int j = 0; j < zz; ++j) {
                    hv[m.vbase[q] + (size_t)k * m.ldv[q] + f.voff[q * P + p] + j] = at(V, p, q, k, j);
                    hu[m.ubase[p] + (size_t)k * m.ldw[p] + f.uoff[p * P + q] + j] = at(U, p, q, k, j);
                }
            for (int j = 0; j < zz; ++j)
                hs[m.sbase[q] + f.voff[q * P + p] + j] = (R)S[(size_t)(p * P + q) * rank + j];
        }
    if (D)
        for (int p = 0; p < P; ++p)
            for (int k = 0; k < Nk; ++k)
                for (int kp = 0; kp < Nk; ++kp) {
                    const size_t e = (((size_t)p * Nk + k) * Nk + kp) * 2;
                    hu[m.ubase[p] + (size_t)k * m.ldw[p] + m.nlr[p] + kp] = make_double2(D[e], D[e + 1]);
                }
    DevBuf tmp;
    tmp.ensure(std::max(hv.size(), hu.size()) * sizeof(double2));
    if (m.vtot > 0) {
        TDAGW_CUDA(cudaMemcpyAsync(tmp.p, hv.data(), hv.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
        launch_convert_in<R>(tmp.as<double2>(), f.V.p, (int64_t)hv.size(), s);
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
    TDAGW_CUDA(cudaMemcpyAsync(tmp.p, hu.data(), hu.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_convert_in<R>(tmp.as<double2>(), f.U.p, (int64_t)hu.size(), s);
    if (!D) ch_fill_diag_from_kernel<R>(c);
    TDAGW_CUDA(cudaMemcpyAsync(f.S.p, hs.data(), hs.size() * sizeof(R), cudaMemcpyHostToDevice, s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
    f.valid = true;
}

template <typename R>
void get_channel_factors(Ctx& c, int* rank, int* ranks, double* U, double* S, double* V, double* D) {
    const HostModel& h = c.hm;
    const int P = h.Nb * h.Nb, Nk = h.Nk;
    ChannelFactors& f = c.ch;
    const ChMeta& m = f.m;
    const int r = f.zmax;
    if (rank) *rank = r;
    if (ranks)
        for (int e = 0; e < P * P; ++e) ranks[e] = f.z[e];
    if (!U && !S && !V && !D) return;
    cudaStream_t s = c.stream;
    DevBuf tmp;
    tmp.ensure((size_t)std::max(m.vtot, m.utot) * sizeof(double2));
    std::vector<double2> hv, hu;
    if (V && m.vtot > 0) {
        hv.resize((size_t)m.vtot);
        launch_convert_out<R>(f.V.p, tmp.as<double2>(), m.vtot, s);
        TDAGW_CUDA(cudaMemcpyAsync(hv.data(), tmp.p, hv.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
    if (U || D) {
        hu.resize((size_t)m.utot);
        launch_convert_out<R>(f.U.p, tmp.as<double2>(), m.utot, s);
        TDAGW_CUDA(cudaMemcpyAsync(hu.data(), tmp.p, hu.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<R> hs((size_t)std::max<long long>(m.stot, 1));
    if (S) {
        TDAGW_CUDA(cudaMemcpyAsync(hs.data(), f.S.p, hs.size() * sizeof(R), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
    const size_t fsz = (size_t)P * P * Nk * r * 2;
    if (U) std::fill(U, U + fsz, 0.0);
    if (V) std::fill(V, V + fsz, 0.0);
    if (S) std::fill(S, S + (size_t)P * P * r, 0.0);
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q) {
            const int zz = f.z[p * P + q];
            if (p == q || zz == 0) continue;
            for (int k = 0; k < Nk; ++k)
                for (int j = 0; j < zz; ++j) {
                    const size_t e = (((size_t)(p * P + q) * Nk + k) * r + j) * 2;
                    if (V) {
                        const double2 v = hv[m.vbase[q] + (size_t)k * m.ldv[q] + f.voff[q * P + p] + j];
                        V[e] = v.x;
                        V[e + 1] = v.y;
                    }
                    if (U) {
                        const double2 u = hu[m.ubase[p] + (size_t)k * m.ldw[p] + f.uoff[p * P + q] + j];
                        U[e] = u.x;
                        U[e + 1] = u.y;
                    }
                }
            if (S)
                for (int j = 0; j < zz; ++j)
                    S[(size_t)(p * P + q) * r + j] = (double)hs[m.sbase[q] + f.voff[q * P + p] + j];
        }
    if (D)
        for (int p = 0; p < P; ++p)
            for (int k = 0; k < Nk; ++k)
                for (int kp = 0; kp < Nk; ++kp) {
                    const double2 d = hu[m.ubase[p] + (size_t)k * m.ldw[p] + m.nlr[p] + kp];
                    const size_t e = (((size_t)p * Nk + k) * Nk + kp) * 2;
                    D[e] = d.x;
                    D[e + 1] = d.y;
                }
}

template <typename R>
void launch_ch_apply(Ctx& c, const void* x, void* y, cudaStream_t s) {
    using C = cplx_t<R>;
    ChannelFactors& f = c.ch;
    const ChMeta& m = f.m;
    const C* xc = static_cast<const C*>(x);
    if (m.stot > 0) {
        const int ns = vpass_splits(m);
        f.part.ensure((size_t)ns * m.stot * sizeof(C));
        dim3 grid((unsigned)((m.stot + 255) / 256), (unsigned)ns);
        ch_vpass_kernel<R><<<grid, 256, 0, s>>>(m, f.V.as<C>(), xc, f.part.as<C>(), ns);
        check_launch("ch_vpass_kernel");
        launch_yreduce<R>(f.part.p, ns, (int)m.stot, f.S.p, f.Y.p, s);
    }
    const int64_t warps = (int64_t)m.P * m.Nk;
    ch_upass_kernel<R><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(
        m, f.U.as<C>(), f.Y.as<C>(), f.gidx.as<int>(), xc, static_cast<C*>(y));
    check_launch("ch_upass_kernel");
}

#define INST(R)                                                                                   \
    template void launch_ch_gather<R>(const Ctx&, int, int, void*, int64_t, cudaStream_t);       \
    template void launch_ch_place<R>(const double2*, int, int, void*, int64_t, int, cudaStream_t); \
    template void ch_fill_diag_from_kernel<R>(Ctx&);                                              \
    template void set_channel_factors<R>(Ctx&, int, const int*, const double*, const double*,    \
                                         const double*, const double*);                          \
    template void get_channel_factors<R>(Ctx&, int*, int*, double*, double*, double*, double*);  \
    template void launch_ch_apply<R>(Ctx&, const void*, void*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace tdagw
