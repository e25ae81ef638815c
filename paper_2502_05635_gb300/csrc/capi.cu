// C ABI of the library (declared in include/tdagw.h): argument checks, buffer ownership,
// the RK4 driver (stage launches, captured into a CUDA graph per chunk of steps) and the
// host <-> device exchange of model, factors, state and observables.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

struct tdagw_ctx {
    tdagw::Ctx c;
};

namespace tdagw {

// message of the last failing call on this thread (tdagw_last_error)
std::string& last_error_message() {
    thread_local std::string msg;
    return msg;
}

namespace {

std::string& g_err_ref() { return last_error_message(); }
#define g_err g_err_ref()

// NVTX range over one entry point: the setup, propagation, adjoint and HHG calls show up by
// name on a profiler's timeline (NVTX is header-only and does nothing without a tool)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

template <class F> int guard(F&& f) {
    try {
        f();
        g_err.clear();
        return TDAGW_OK;
    } catch (const Error& e) {
        g_err = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return TDAGW_ERR_OOM;
    } catch (const std::exception& e) {
        g_err = e.what();
        return TDAGW_ERR_CUDA;
    } catch (...) {
        g_err = "unknown error";
        return TDAGW_ERR_CUDA;
    }
}

void require_built(const Ctx& c) {
    TDAGW_REQUIRE(c.built, TDAGW_ERR_NOT_BUILT, "tdagw_build_kernel has not been called");
}

template <typename R> void upload_c128(DevBuf& dst, const std::vector<zd>& src, cudaStream_t s) {
    const int64_t n = (int64_t)src.size();
    DevBuf tmp;
    tmp.ensure(n * sizeof(double2));
    TDAGW_CUDA(cudaMemcpyAsync(tmp.p, src.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s));
    dst.ensure(n * sizeof(cplx_t<R>));
    launch_convert_in<R>(tmp.as<double2>(), dst.p, n, s);
    TDAGW_CUDA(cudaStreamSynchronize(s));
}

template <typename R> void build(Ctx& c) {
    cudaStream_t s = c.stream;
    build_host_model(c.desc, c.hm);
    const HostModel& h = c.hm;
    const int64_t N = h.N;
    upload_c128<R>(c.dx, h.dx, s);
    upload_c128<R>(c.dy, h.dy, s);
    upload_c128<R>(c.vx, h.vx, s);
    // band-gap table eps_n - eps_m per pair element: (hi, lo) floats or doubles
    if (sizeof(R) == 4) {
        std::vector<float2> g(N);
        for (int k = 0; k < h.Nk; ++k)
            for (int n = 0; n < h.Nb; ++n)
                for (int m = 0; m < h.Nb; ++m) {
                    const double d = h.eps[(size_t)k * h.Nb + n] - h.eps[(size_t)k * h.Nb + m];
                    const float hi = (float)d;
                    g[((size_t)k * h.Nb + n) * h.Nb + m] = make_float2(hi, (float)(d - (double)hi));
                }
        c.gap.ensure(N * sizeof(float2));
        TDAGW_CUDA(cudaMemcpyAsync(c.gap.p, g.data(), N * sizeof(float2), cudaMemcpyHostToDevice, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    } else {
        std::vector<double> g(N);
        for (int k = 0; k < h.Nk; ++k)
            for (int n = 0; n < h.Nb; ++n)
                for (int m = 0; m < h.Nb; ++m)
                    g[((size_t)k * h.Nb + n) * h.Nb + m] =
                        h.eps[(size_t)k * h.Nb + n] - h.eps[(size_t)k * h.Nb + m];
        c.gap.ensure(N * sizeof(double));
        TDAGW_CUDA(cudaMemcpyAsync(c.gap.p, g.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
    c.Ud.ensure(h.U.size() * sizeof(double2));
    TDAGW_CUDA(cudaMemcpyAsync(c.Ud.p, h.U.data(), h.U.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    c.Wd.ensure(h.Wtab.size() * sizeof(double));
    TDAGW_CUDA(cudaMemcpyAsync(c.Wd.p, h.Wtab.data(), h.Wtab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    if (!h.Mx.empty()) {
        c.Mxd.ensure(h.Mx.size() * sizeof(double2));
        c.vGd.ensure(8 * sizeof(double));
        TDAGW_CUDA(cudaMemcpyAsync(c.Mxd.p, h.Mx.data(), h.Mx.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
        TDAGW_CUDA(cudaMemcpyAsync(c.vGd.p, h.vG, 8 * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    c.K.ensure((size_t)N * (size_t)N * sizeof(cplx_t<R>));
    launch_build_kernel<R>(c, s);
    // diag(K): every (N+1)-th element
    c.diagK.ensure(N * sizeof(cplx_t<R>));
    TDAGW_CUDA(cudaMemcpy2DAsync(c.diagK.p, sizeof(cplx_t<R>), c.K.p, (N + 1) * sizeof(cplx_t<R>),
                                 sizeof(cplx_t<R>), N, cudaMemcpyDeviceToDevice, s));
    // propagation buffers
    for (DevBuf* b : {&c.Ssum, &c.Ccomp, &c.X, &c.acc, &c.dS}) {
        b->ensure(N * sizeof(cplx_t<R>));
        TDAGW_CUDA(cudaMemsetAsync(b->p, 0, N * sizeof(cplx_t<R>), s));
    }
    const int64_t blocks = (N + 255) / 256;
    c.red.ensure(blocks * 3 * sizeof(double));
    c.counter.ensure(sizeof(unsigned));
    TDAGW_CUDA(cudaMemsetAsync(c.counter.p, 0, sizeof(unsigned), s));
    c.stepctr.ensure(sizeof(int64_t));
    TDAGW_CUDA(cudaStreamSynchronize(s));
    c.step = 0;
    c.built = true;
}

template <typename R> void set_factors(Ctx& c, int r, const double* U, const double* S,
                                       const double* V, const double* diag) {
    using C = cplx_t<R>;
    cudaStream_t s = c.stream;
    const int64_t N = c.hm.N;
    const int64_t ldu = r + (r & 1);
    // U and V: N x ldu row-major (padded, zero pad column)
    std::vector<double2> hu((size_t)N * ldu, make_double2(0, 0)), hv((size_t)N * ldu, make_double2(0, 0));
    for (int64_t i = 0; i < N; ++i)
        for (int j = 0; j < r; ++j) {
            hu[(size_t)i * ldu + j] = make_double2(U[2 * (i * r + j)], U[2 * (i * r + j) + 1]);
            hv[(size_t)i * ldu + j] = make_double2(V[2 * (i * r + j)], V[2 * (i * r + j) + 1]);
        }
    DevBuf tmp;
    tmp.ensure(hu.size() * sizeof(double2));
    c.U.ensure(hu.size() * sizeof(C));
    TDAGW_CUDA(cudaMemcpyAsync(tmp.p, hu.data(), hu.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_convert_in<R>(tmp.as<double2>(), c.U.p, (int64_t)hu.size(), s);
    TDAGW_CUDA(cudaStreamSynchronize(s));
    c.V.ensure(hv.size() * sizeof(C));
    TDAGW_CUDA(cudaMemcpyAsync(tmp.p, hv.data(), hv.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_convert_in<R>(tmp.as<double2>(), c.V.p, (int64_t)hv.size(), s);
    TDAGW_CUDA(cudaStreamSynchronize(s));
    std::vector<R> hs(r);
    for (int j = 0; j < r; ++j) hs[j] = (R)S[j];
    c.S.ensure(r * sizeof(R));
    TDAGW_CUDA(cudaMemcpyAsync(c.S.p, hs.data(), r * sizeof(R), cudaMemcpyHostToDevice, s));
    if (c.kdiag) {
        // the k = k' blocks: Nk x P x P
        const int64_t nb = (int64_t)c.hm.Nk * c.hm.Nb * c.hm.Nb * c.hm.Nb * c.hm.Nb;
        c.kblkF.ensure(nb * sizeof(C));
        if (diag) {
            DevBuf t2;
            t2.ensure(nb * sizeof(double2));
            TDAGW_CUDA(cudaMemcpyAsync(t2.p, diag, nb * sizeof(double2), cudaMemcpyHostToDevice, s));
            launch_convert_in<R>(t2.as<double2>(), c.kblkF.p, nb, s);
            TDAGW_CUDA(cudaStreamSynchronize(s));
        } else {
            launch_gather_kblocks<R>(c, c.kblkF.p, s);
        }
    }
    c.diagF.ensure(N * sizeof(C));
    if (diag && !c.kdiag) {
        TDAGW_CUDA(cudaMemcpyAsync(tmp.p, diag, N * sizeof(double2), cudaMemcpyHostToDevice, s));
        launch_convert_in<R>(tmp.as<double2>(), c.diagF.p, N, s);
    } else {
        TDAGW_CUDA(cudaMemcpyAsync(c.diagF.p, c.diagK.p, N * sizeof(C), cudaMemcpyDeviceToDevice, s));
    }
    c.rank = r;
    c.ysplit = choose_ysplit(r, N);
    c.ypart.ensure((size_t)c.ysplit * r * sizeof(C));
    c.ytil.ensure((size_t)ldu * sizeof(C));
    TDAGW_CUDA(cudaMemsetAsync(c.ytil.p, 0, ldu * sizeof(C), s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
}

template <typename R> void get_factors(Ctx& c, double* U, double* S, double* V, double* diag) {
    using C = cplx_t<R>;
    cudaStream_t s = c.stream;
    const int64_t N = c.hm.N, r = c.rank, ldu = r + (r & 1);
    DevBuf tmp;
    tmp.ensure((size_t)N * ldu * sizeof(double2));
    std::vector<double2> h((size_t)N * ldu);
    for (int which = 0; which < 2; ++which) {
        double* out = which == 0 ? U : V;
        if (!out) continue;
        launch_convert_out<R>(which == 0 ? c.U.p : c.V.p, tmp.as<double2>(), N * ldu, s);
        TDAGW_CUDA(cudaMemcpyAsync(h.data(), tmp.p, N * ldu * sizeof(double2), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = 0; j < r; ++j) {
                out[2 * (i * r + j)] = h[i * ldu + j].x;
                out[2 * (i * r + j) + 1] = h[i * ldu + j].y;
            }
    }
    if (S) {
        std::vector<R> hs(r);
        TDAGW_CUDA(cudaMemcpyAsync(hs.data(), c.S.p, r * sizeof(R), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
        for (int64_t j = 0; j < r; ++j) S[j] = (double)hs[j];
    }
    if (diag && c.kdiag) {
        const int64_t nb = (int64_t)c.hm.Nk * c.hm.Nb * c.hm.Nb * c.hm.Nb * c.hm.Nb;
        DevBuf t2;
        t2.ensure(nb * sizeof(double2));
        launch_convert_out<R>(c.kblkF.p, t2.as<double2>(), nb, s);
        TDAGW_CUDA(cudaMemcpyAsync(diag, t2.p, nb * sizeof(double2), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    } else if (diag) {
        launch_convert_out<R>(c.diagF.p, tmp.as<double2>(), N, s);
        TDAGW_CUDA(cudaMemcpyAsync(diag, tmp.p, N * sizeof(double2), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    }
}

// y = K x (full), diag o x + U (S o (V^H x)) (low-rank) or the channel-wise form: the
// kernel contraction of one RK4 stage (Eq. sigma-from-k / Eq. svd_acc / Eq. svd-channel-wise).
template <typename R> void apply(Ctx& c, int mode, const void* x, void* y, cudaStream_t s) {
    const int64_t N = c.hm.N;
    if (mode == TDAGW_FULL) {
        launch_gemv<R>(c.K.p, N, N, N, x, y, 1, nullptr, nullptr, s);
    } else if (mode == TDAGW_CHANNEL) {
        launch_ch_apply<R>(c, x, y, s);
    } else {
        const int r = c.rank;
        const int64_t ldu = r + (r & 1);
        launch_vcols<R>(c.V.p, ldu, N, r, x, c.ypart.p, c.ysplit, s);
        launch_yreduce<R>(c.ypart.p, c.ysplit, r, c.S.p, c.ytil.p, s);
        if (c.kdiag) {
            launch_gemv<R>(c.U.p, ldu, N, r, c.ytil.p, y, 1, nullptr, nullptr, s);
            launch_kblock_add<R>(c.kblkF.p, x, y, c.hm.Nk, c.hm.Nb * c.hm.Nb, s);
        } else {
            launch_gemv<R>(c.U.p, ldu, N, r, c.ytil.p, y, 1, c.diagF.p, x, s);
        }
    }
}

template <typename R> void one_step(Ctx& c, int mode, double dt, double dirx, double diry,
                                    bool kahan, cudaStream_t s) {
    for (int st = 0; st < 4; ++st) {
        apply<R>(c, mode, c.X.p, c.dS.p, s);
        launch_stage<R>(c, st, dt, dirx, diry, kahan, s);
    }
}

template <typename R> void propagate(Ctx& c, const tdagw_field& f, int T, double dt, int mode,
                                     int flags) {
    cudaStream_t s = c.stream;
    const int64_t N = c.hm.N;
    using C = cplx_t<R>;
    if (flags & TDAGW_FLAG_RESET) {
        for (DevBuf* b : {&c.Ssum, &c.Ccomp, &c.X})
            TDAGW_CUDA(cudaMemsetAsync(b->p, 0, N * sizeof(C), s));
        c.step = 0;
    }
    const int64_t nsamp = 2 * (int64_t)T + 1;
    c.Etab.ensure(nsamp * sizeof(double));
    if (f.kind == TDAGW_FIELD_TABLE) {
        TDAGW_CUDA(cudaMemcpyAsync(c.Etab.p, f.table, nsamp * sizeof(double), cudaMemcpyHostToDevice, s));
    } else {
        launch_field_table(f, (double)c.step * dt, dt, nsamp, c.Etab.as<double>(), s);
    }
    c.obs.ensure((T + 1) * 3 * sizeof(double));
    launch_observables_row<R>(c, c.X.p, 0, s);
    TDAGW_CUDA(cudaMemsetAsync(c.stepctr.p, 0, sizeof(int64_t), s));
    const bool kahan = !(flags & TDAGW_FLAG_NO_KAHAN);
    const double dirx = f.dir_x, diry = f.dir_y;
    int done = 0;
    const bool test_timeout = (flags & TDAGW_FLAG_TEST_TIMEOUT) != 0;
    if (mode == TDAGW_LOWRANK && !(flags & TDAGW_FLAG_STAGEWISE) && T > 0 &&
        launch_lr_persistent(c, T, dt, dirx, diry, kahan, test_timeout, s))
        done = T;
    if (mode == TDAGW_CHANNEL && !(flags & TDAGW_FLAG_STAGEWISE) && T > 0 &&
        launch_ch_persistent(c, T, dt, dirx, diry, kahan, test_timeout, s))
        done = T;
    if (!(flags & TDAGW_FLAG_NO_GRAPH) && T - done >= 2) {
        const int G = std::min(T, 32);
        cudaGraph_t g = nullptr;
        if (!c.cap) TDAGW_CUDA(cudaStreamCreateWithFlags(&c.cap, cudaStreamNonBlocking));
        TDAGW_CUDA(cudaStreamBeginCapture(c.cap, cudaStreamCaptureModeThreadLocal));
        try {
            for (int q = 0; q < G; ++q) one_step<R>(c, mode, dt, dirx, diry, kahan, c.cap);
        } catch (...) {
            cudaStreamEndCapture(c.cap, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        TDAGW_CUDA(cudaStreamEndCapture(c.cap, &g));
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        TDAGW_CUDA(e);
        const int reps = T / G;
        cudaError_t le = cudaSuccess;
        for (int q = 0; q < reps && le == cudaSuccess; ++q) le = cudaGraphLaunch(ge, s);
        cudaGraphExecDestroy(ge);
        TDAGW_CUDA(le);
        done = reps * G;
    }
    for (; done < T; ++done) one_step<R>(c, mode, dt, dirx, diry, kahan, s);
    c.step += T;
    c.obs_rows = T + 1;
}

template <typename R> void get_state(Ctx& c, double* drho, double* carry) {
    cudaStream_t s = c.stream;
    const int64_t N = c.hm.N;
    DevBuf t1, t2;
    t1.ensure(N * sizeof(double2));
    t2.ensure(N * sizeof(double2));
    launch_convert_out<R>(c.Ssum.p, t1.as<double2>(), N, s);
    launch_convert_out<R>(c.Ccomp.p, t2.as<double2>(), N, s);
    std::vector<double> a(2 * N), b(2 * N);
    TDAGW_CUDA(cudaMemcpyAsync(a.data(), t1.p, N * sizeof(double2), cudaMemcpyDeviceToHost, s));
    TDAGW_CUDA(cudaMemcpyAsync(b.data(), t2.p, N * sizeof(double2), cudaMemcpyDeviceToHost, s));
    TDAGW_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < 2 * N; ++i) {
        if (drho) drho[i] = a[i] + b[i];
        if (carry) carry[i] = b[i];
    }
}

template <typename R> void set_state(Ctx& c, const double* drho, const double* carry) {
    cudaStream_t s = c.stream;
    const int64_t N = c.hm.N;
    std::vector<double> hs(2 * N), hc(2 * N, 0.0);
    for (int64_t i = 0; i < 2 * N; ++i) {
        hc[i] = carry ? carry[i] : 0.0;
        hs[i] = drho[i] - hc[i];
    }
    DevBuf t;
    t.ensure(N * sizeof(double2));
    TDAGW_CUDA(cudaMemcpyAsync(t.p, hs.data(), N * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_convert_in<R>(t.as<double2>(), c.Ssum.p, N, s);
    TDAGW_CUDA(cudaStreamSynchronize(s));
    TDAGW_CUDA(cudaMemcpyAsync(t.p, hc.data(), N * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_convert_in<R>(t.as<double2>(), c.Ccomp.p, N, s);
    TDAGW_CUDA(cudaStreamSynchronize(s));
    TDAGW_CUDA(cudaMemcpyAsync(t.p, drho, N * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_convert_in<R>(t.as<double2>(), c.X.p, N, s);
    TDAGW_CUDA(cudaStreamSynchronize(s));
}

// After a synchronisation: report (and clear) the error word of a persistent launch.
void check_device_error(Ctx& c) {
    if (!c.persistent_launched || !c.sync.p) return;
    int err = 0;
    TDAGW_CUDA(cudaMemcpy(&err, c.sync.as<unsigned>() + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        TDAGW_CUDA(cudaMemset(c.sync.as<unsigned>() + 2, 0, sizeof(int)));
        c.persistent_launched = false;
        throw Error(TDAGW_ERR_TIMEOUT, "a bounded device-side wait of the propagation gave up");
    }
}

void check_desc(const tdagw_model_desc* d) {
    TDAGW_REQUIRE(d, TDAGW_ERR_INVALID_ARG, "desc is NULL");
    TDAGW_REQUIRE(d->L >= 1 && d->L <= 4096, TDAGW_ERR_INVALID_ARG, "L must be in [1, 4096]");
    TDAGW_REQUIRE(d->nb_copies == 1 || d->nb_copies == 2, TDAGW_ERR_INVALID_ARG,
                  "nb_copies must be 1 or 2");
    TDAGW_REQUIRE(d->dtype == TDAGW_C64 || d->dtype == TDAGW_C128, TDAGW_ERR_INVALID_ARG,
                  "dtype must be TDAGW_C64 or TDAGW_C128");
    TDAGW_REQUIRE(d->a > 0 && d->r0 > 0 && d->Delta > 0, TDAGW_ERR_INVALID_ARG,
                  "a, r0 and Delta must be positive");
    TDAGW_REQUIRE(d->exchange >= 0.0 && d->exchange < 1e6, TDAGW_ERR_INVALID_ARG,
                  "exchange must be in [0, 1e6)");
}

}  // namespace
}  // namespace tdagw

using namespace tdagw;

#define DISPATCH(ctx, fn, ...)                                                             \
    ((ctx)->c.dtype == TDAGW_C64 ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

extern "C" {

int tdagw_create(const tdagw_model_desc* desc, void* stream, tdagw_ctx** out) {
    return guard([&] {
        TDAGW_REQUIRE(out, TDAGW_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        check_desc(desc);
        std::unique_ptr<tdagw_ctx> h(new tdagw_ctx());
        h->c.desc = *desc;
        h->c.dtype = desc->dtype;
        h->c.csz = desc->dtype == TDAGW_C64 ? 8 : 16;
        h->c.stream = static_cast<cudaStream_t>(stream);  // NULL: legacy default stream
        *out = h.release();
    });
}

int tdagw_build_kernel(tdagw_ctx* ctx) {
    const Range nv("tdagw_build_kernel");
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        DISPATCH(ctx, build, ctx->c);
    });
}

int tdagw_model_info(const tdagw_ctx* ctx, int64_t* N, int* Nb, int* Nk) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        const tdagw_model_desc& d = ctx->c.desc;
        const int nb = 2 * d.nb_copies, nk = d.L * d.L;
        if (N) *N = (int64_t)nb * nb * nk;
        if (Nb) *Nb = nb;
        if (Nk) *Nk = nk;
    });
}

int tdagw_get_model(const tdagw_ctx* ctx, double* eps, double* dx, double* dy, double* vx,
                    double* U) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        require_built(ctx->c);
        const HostModel& h = ctx->c.hm;
        if (eps) std::memcpy(eps, h.eps.data(), h.eps.size() * sizeof(double));
        if (dx) std::memcpy(dx, h.dx.data(), h.dx.size() * sizeof(zd));
        if (dy) std::memcpy(dy, h.dy.data(), h.dy.size() * sizeof(zd));
        if (vx) std::memcpy(vx, h.vx.data(), h.vx.size() * sizeof(zd));
        if (U) std::memcpy(U, h.U.data(), h.U.size() * sizeof(zd));
    });
}

int tdagw_get_kernel_entries(tdagw_ctx* ctx, const int64_t* rows, const int64_t* cols,
                             int64_t n, double* out) {
    return guard([&] {
        TDAGW_REQUIRE(ctx && rows && cols && out && n >= 0, TDAGW_ERR_INVALID_ARG, "bad arguments");
        require_built(ctx->c);
        const int64_t N = ctx->c.hm.N;
        for (int64_t i = 0; i < n; ++i)
            TDAGW_REQUIRE(rows[i] >= 0 && rows[i] < N && cols[i] >= 0 && cols[i] < N,
                          TDAGW_ERR_INVALID_ARG, "entry index out of range");
        if (n == 0) return;
        cudaStream_t s = ctx->c.stream;
        DevBuf ri, ci, o;
        ri.ensure(n * sizeof(int64_t));
        ci.ensure(n * sizeof(int64_t));
        o.ensure(n * sizeof(double2));
        TDAGW_CUDA(cudaMemcpyAsync(ri.p, rows, n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        TDAGW_CUDA(cudaMemcpyAsync(ci.p, cols, n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DISPATCH(ctx, launch_gather_entries, ctx->c, ri.as<int64_t>(), ci.as<int64_t>(), n,
                 o.as<double2>(), s);
        TDAGW_CUDA(cudaMemcpyAsync(out, o.p, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
        TDAGW_CUDA(cudaStreamSynchronize(s));
    });
}

int tdagw_compress_svd(tdagw_ctx* ctx, int rank, int oversample, int power_iters,
                       uint64_t seed, int precision) {
    const Range nv("tdagw_compress_svd");
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        require_built(ctx->c);
        TDAGW_REQUIRE(rank >= 1 && oversample >= 0 && power_iters >= 0 &&
                          (int64_t)rank + oversample <= ctx->c.hm.N,
                      TDAGW_ERR_INVALID_ARG, "need 1 <= rank and rank + oversample <= N");
        TDAGW_REQUIRE(precision == 0 || precision == 1, TDAGW_ERR_INVALID_ARG, "precision must be 0 or 1");
        TDAGW_REQUIRE(precision == 0 || ctx->c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED,
                      "split-FP16 factors need a complex64 context");
        TDAGW_REQUIRE(precision == 0 || !ctx->c.kdiag, TDAGW_ERR_UNSUPPORTED,
                      "split-FP16 factors need the strict-diagonal reading of K^diag");
        ctx->c.tc_valid = false;
        if (ctx->c.kdiag) {
            const HostModel& h = ctx->c.hm;
            ctx->c.kblkF.ensure((size_t)h.Nk * h.Nb * h.Nb * h.Nb * h.Nb * ctx->c.csz);
            if (ctx->c.dtype == TDAGW_C64)
                launch_gather_kblocks<float>(ctx->c, ctx->c.kblkF.p, ctx->c.stream);
            else
                launch_gather_kblocks<double>(ctx->c, ctx->c.kblkF.p, ctx->c.stream);
        }
        DISPATCH(ctx, rsvd_compress, ctx->c, rank, oversample, power_iters, seed);
        if (precision == 1) pack_factors_tc(ctx->c);
    });
}

int tdagw_set_factors(tdagw_ctx* ctx, int rank, const double* U, const double* S,
                      const double* V, const double* diag) {
    return guard([&] {
        TDAGW_REQUIRE(ctx && U && S && V, TDAGW_ERR_INVALID_ARG, "NULL argument");
        require_built(ctx->c);
        TDAGW_REQUIRE(rank >= 1 && rank <= ctx->c.hm.N, TDAGW_ERR_INVALID_ARG, "rank out of range");
        ctx->c.tc_valid = false;
        DISPATCH(ctx, set_factors, ctx->c, rank, U, S, V, diag);
    });
}

int tdagw_get_factors(tdagw_ctx* ctx, int* rank, double* U, double* S, double* V, double* diag) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        if (rank) *rank = ctx->c.rank;
        if (!U && !S && !V && !diag) return;
        TDAGW_REQUIRE(ctx->c.rank > 0, TDAGW_ERR_NO_FACTORS, "no factors installed");
        DISPATCH(ctx, get_factors, ctx->c, U, S, V, diag);
    });
}

int tdagw_set_kdiag_blocks(tdagw_ctx* ctx, int on) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        TDAGW_REQUIRE(on == 0 || on == 1, TDAGW_ERR_INVALID_ARG, "on must be 0 or 1");
        Ctx& c = ctx->c;
        if (c.kdiag != on) {
            c.kdiag = on;
            c.rank = 0;        // installed factors split K the other way
            c.tc_valid = false;
        }
    });
}

int tdagw_compress_channels(tdagw_ctx* ctx, int rank, int oversample, int power_iters,
                            uint64_t seed, double rel_tol) {
    const Range nv("tdagw_compress_channels");
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        require_built(ctx->c);
        TDAGW_REQUIRE(rank >= 0 && rank <= ctx->c.hm.Nk && oversample >= 0 && power_iters >= 0 &&
                          rel_tol >= 0.0,
                      TDAGW_ERR_INVALID_ARG, "need 0 <= rank <= Nk, oversample, power_iters, rel_tol >= 0");
        DISPATCH(ctx, rsvd_channels, ctx->c, rank, oversample, power_iters, seed, rel_tol);
    });
}

int tdagw_set_channel_factors(tdagw_ctx* ctx, int rank, const int* ranks, const double* U,
                              const double* S, const double* V, const double* D) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        require_built(ctx->c);  // the channel layout takes Nb and Nk from the built model
        TDAGW_REQUIRE(rank >= 0 && rank <= ctx->c.hm.Nk, TDAGW_ERR_INVALID_ARG, "need 0 <= rank <= Nk");
        TDAGW_REQUIRE(rank == 0 || (U && S && V), TDAGW_ERR_INVALID_ARG, "NULL factor array");
        DISPATCH(ctx, set_channel_factors, ctx->c, rank, ranks, U, S, V, D);
    });
}

int tdagw_get_channel_factors(tdagw_ctx* ctx, int* rank, int* ranks, double* U, double* S, double* V,
                              double* D) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        const bool any = ranks || U || S || V || D;
        if (!ctx->c.ch.valid) {
            if (rank) *rank = 0;
            TDAGW_REQUIRE(!any, TDAGW_ERR_NO_FACTORS, "no channel factors installed");
            return;
        }
        DISPATCH(ctx, get_channel_factors, ctx->c, rank, ranks, U, S, V, D);
    });
}

int tdagw_apply(tdagw_ctx* ctx, int mode, const void* x, void* y) {
    return guard([&] {
        TDAGW_REQUIRE(ctx && x && y, TDAGW_ERR_INVALID_ARG, "NULL argument");
        require_built(ctx->c);
        TDAGW_REQUIRE(mode == TDAGW_FULL || mode == TDAGW_LOWRANK || mode == TDAGW_CHANNEL,
                      TDAGW_ERR_INVALID_ARG, "bad mode");
        TDAGW_REQUIRE(mode != TDAGW_LOWRANK || ctx->c.rank > 0, TDAGW_ERR_NO_FACTORS, "no factors");
        TDAGW_REQUIRE(mode != TDAGW_CHANNEL || ctx->c.ch.valid, TDAGW_ERR_NO_FACTORS, "no channel factors");
        TDAGW_REQUIRE(((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0), TDAGW_ERR_INVALID_ARG,
                      "x and y must be 16-byte aligned");
        TDAGW_REQUIRE(x != y, TDAGW_ERR_INVALID_ARG, "x and y must not alias");
        DISPATCH(ctx, apply, ctx->c, mode, x, y, ctx->c.stream);
    });
}

int tdagw_propagate(tdagw_ctx* ctx, const tdagw_field* fields, int B, const int* steps,
                    double dt, int mode, int flags) {
    const Range nv("tdagw_propagate");
    return guard([&] {
        TDAGW_REQUIRE(ctx && fields && steps, TDAGW_ERR_INVALID_ARG, "NULL argument");
        require_built(ctx->c);
        TDAGW_REQUIRE(B >= 1 && B <= 65536, TDAGW_ERR_INVALID_ARG, "B must be in [1, 65536]");
        for (int b = 0; b < B; ++b)
            TDAGW_REQUIRE(steps[b] >= 0 && steps[b] <= (1 << 26), TDAGW_ERR_INVALID_ARG, "bad step count");
        TDAGW_REQUIRE(dt > 0 && dt < 1e6, TDAGW_ERR_INVALID_ARG, "bad dt");
        TDAGW_REQUIRE(mode == TDAGW_FULL || mode == TDAGW_LOWRANK || mode == TDAGW_CHANNEL,
                      TDAGW_ERR_INVALID_ARG, "bad mode");
        TDAGW_REQUIRE(mode != TDAGW_LOWRANK || ctx->c.rank > 0, TDAGW_ERR_NO_FACTORS,
                      "low-rank mode needs factors (tdagw_compress_svd or tdagw_set_factors)");
        TDAGW_REQUIRE(mode != TDAGW_CHANNEL || ctx->c.ch.valid, TDAGW_ERR_NO_FACTORS,
                      "channel mode needs channel factors (tdagw_compress_channels or "
                      "tdagw_set_channel_factors)");
        TDAGW_REQUIRE(mode != TDAGW_CHANNEL || !(flags & TDAGW_FLAG_CHECKPOINT), TDAGW_ERR_UNSUPPORTED,
                      "channel mode runs without checkpoints");
        for (int b = 0; b < B; ++b) {
            const tdagw_field& f = fields[b];
            TDAGW_REQUIRE(f.kind >= 0 && f.kind <= 3, TDAGW_ERR_INVALID_ARG, "bad field kind");
            TDAGW_REQUIRE(f.kind != TDAGW_FIELD_TABLE || f.table, TDAGW_ERR_INVALID_ARG,
                          "table field without samples");
            TDAGW_REQUIRE(f.kind != TDAGW_FIELD_GAUSS_COS || f.sigma > 0, TDAGW_ERR_INVALID_ARG,
                          "sigma must be positive");
            TDAGW_REQUIRE(f.kind != TDAGW_FIELD_SIN2_SIN || f.T_pulse > 0, TDAGW_ERR_INVALID_ARG,
                          "T_pulse must be positive");
        }
        TDAGW_REQUIRE(!(flags & TDAGW_FLAG_SPLIT_F16) || mode == TDAGW_LOWRANK || mode == TDAGW_CHANNEL,
                      TDAGW_ERR_INVALID_ARG, "TDAGW_FLAG_SPLIT_F16 applies to the low-rank and channel-wise kernels");
        TDAGW_REQUIRE(mode != TDAGW_LOWRANK || !ctx->c.kdiag || !(flags & TDAGW_FLAG_SPLIT_F16),
                      TDAGW_ERR_UNSUPPORTED, "split-FP16 factors need the strict-diagonal reading of K^diag");
        if (flags & TDAGW_FLAG_SPLIT_F16) {
            int tmax = 0;
            for (int b = 0; b < B; ++b) tmax = std::max(tmax, steps[b]);
            TDAGW_REQUIRE(tmax > 0, TDAGW_ERR_INVALID_ARG, "at least one trajectory needs steps");
            if (mode == TDAGW_CHANNEL)
                propagate_channel_tc(ctx->c, fields, B, steps, dt, flags);
            else
                propagate_batched_tc(ctx->c, fields, B, steps, dt, flags);
        } else if (B == 1 && !(flags & TDAGW_FLAG_CHECKPOINT)) {
            DISPATCH(ctx, propagate, ctx->c, fields[0], steps[0], dt, mode, flags);
            ctx->c.obs_B = 1;
            ctx->c.adj.valid = false;
        } else {
            int tmax = 0;
            for (int b = 0; b < B; ++b) tmax = std::max(tmax, steps[b]);
            TDAGW_REQUIRE(tmax > 0, TDAGW_ERR_INVALID_ARG, "at least one trajectory needs steps");
            propagate_batched(ctx->c, fields, B, steps, dt, mode, flags);
        }
    });
}

int tdagw_adjoint(tdagw_ctx* ctx, const double* dJdobs, double* dJdE, double* dJdparams) {
    const Range nv("tdagw_adjoint");
    return guard([&] {
        TDAGW_REQUIRE(ctx && dJdobs, TDAGW_ERR_INVALID_ARG, "NULL argument");
        require_built(ctx->c);
        TDAGW_REQUIRE(ctx->c.dtype == TDAGW_C64, TDAGW_ERR_UNSUPPORTED, "the adjoint needs a complex64 context");
        adjoint_batched(ctx->c, dJdobs, dJdE, dJdparams);
    });
}

int tdagw_observables(tdagw_ctx* ctx, double* out, int64_t max_rows, int64_t* rows, int host) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        if (rows) *rows = ctx->c.obs_rows;
        if (!out) return;
        const int64_t n = std::min<int64_t>(max_rows, ctx->c.obs_rows);
        if (n <= 0) return;
        cudaStream_t s = ctx->c.stream;
        TDAGW_CUDA(cudaMemcpyAsync(out, ctx->c.obs.p, n * ctx->c.obs_B * 3 * sizeof(double),
                                   host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        if (host) {
            TDAGW_CUDA(cudaStreamSynchronize(s));
            check_device_error(ctx->c);
        }
    });
}

int tdagw_get_state(tdagw_ctx* ctx, double* drho, double* carry, int64_t* step) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        require_built(ctx->c);
        if (step) *step = ctx->c.step;
        if (drho || carry) DISPATCH(ctx, get_state, ctx->c, drho, carry);
        check_device_error(ctx->c);
    });
}

int tdagw_set_state(tdagw_ctx* ctx, const double* drho, const double* carry, int64_t step) {
    return guard([&] {
        TDAGW_REQUIRE(ctx && drho && step >= 0, TDAGW_ERR_INVALID_ARG, "bad arguments");
        require_built(ctx->c);
        DISPATCH(ctx, set_state, ctx->c, drho, carry);
        ctx->c.step = step;
    });
}

int tdagw_hhg_spectrum(const double* J, int64_t rows, int64_t stride, int B, const int* steps, double dt,
                       const double* omega, int nfreq, double* out, void* stream) {
    const Range nv("tdagw_hhg_spectrum");
    return guard([&] {
        TDAGW_REQUIRE(J && steps && omega && out, TDAGW_ERR_INVALID_ARG, "NULL argument");
        TDAGW_REQUIRE(B >= 1 && nfreq >= 1 && stride >= 1 && rows >= 1 && dt > 0, TDAGW_ERR_INVALID_ARG,
                      "need B, nfreq, stride, rows >= 1 and dt > 0");
        TDAGW_REQUIRE(B <= 65535, TDAGW_ERR_INVALID_ARG, "B must be at most 65535");
        for (int b = 0; b < B; ++b) TDAGW_REQUIRE(steps[b] >= 0, TDAGW_ERR_INVALID_ARG, "negative step count");
        hhg_spectrum(J, rows, stride, B, steps, dt, omega, nfreq, out, static_cast<cudaStream_t>(stream));
    });
}

int tdagw_sync(tdagw_ctx* ctx) {
    return guard([&] {
        TDAGW_REQUIRE(ctx, TDAGW_ERR_INVALID_ARG, "ctx is NULL");
        TDAGW_CUDA(cudaStreamSynchronize(ctx->c.stream));
        check_device_error(ctx->c);
    });
}

const char* tdagw_last_error(void) { return g_err.c_str(); }

void tdagw_destroy(tdagw_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->c.stream);
    delete ctx;
}

}  // extern "C"

#ifdef TDAGW_TRACE
// traced builds only: CUDA graphs cached for batched launches (-1: capture unavailable)
extern "C" int tdagw_debug_batch_graphs(tdagw_ctx* ctx) {
    return ctx->c.batch_graphs_off ? -1 : (int)ctx->c.batch_graphs.size();
}
#endif
