// Shared definitions of the TD-aGW CUDA library: complex arithmetic on float2/double2,
// error handling, device buffers and the context object behind the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <map>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "tdagw.h"

namespace tdagw {

// ------------------------------------------------------------------ errors -----------

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define TDAGW_CUDA(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            throw ::tdagw::Error(e_ == cudaErrorMemoryAllocation ? TDAGW_ERR_OOM           \
                                                                 : TDAGW_ERR_CUDA,         \
                                 std::string(#call) + ": " + cudaGetErrorString(e_));      \
        }                                                                                  \
    } while (0)

#define TDAGW_REQUIRE(cond, code, msg)                                                     \
    do {                                                                                   \
        if (!(cond)) throw ::tdagw::Error((code), (msg));                                  \
    } while (0)

// message of the last failing call on this thread (returned by tdagw_last_error)
std::string& last_error_message();

inline void check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        throw Error(TDAGW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ complex ----------

template <typename R> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename R> using cplx_t = typename Cplx<R>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
    return mk(a.x * s, a.y * s);
}
// acc + a * b (complex fused multiply-add, 4 real FMAs)
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cfmac(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

// ------------------------------------------------------------------ buffers ----------

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void ensure(size_t b) {
        if (b <= bytes && p) return;
        release();
        if (b == 0) return;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            throw Error(e == cudaErrorMemoryAllocation ? TDAGW_ERR_OOM : TDAGW_ERR_CUDA,
                        "cudaMalloc(" + std::to_string(b) + " B): " + cudaGetErrorString(e));
        }
        bytes = b;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------ host model -------

using zd = std::complex<double>;

struct HostModel {
    int L = 0, Nb = 0, Nk = 0, norb = 0;
    int64_t N = 0;
    std::vector<double> eps;     // Nk * Nb
    std::vector<zd> U;           // Nk * norb * Nb (column n = band n)
    std::vector<zd> dx, dy, vx;  // Nk * Nb * Nb
    std::vector<double> Wtab;    // L * L, W at grid offset (di, dj) (minimum image), W0 at 0
    double W0 = 0.0;
    // exchange term (lambda_x > 0 only): M_nm(k, G) for the eight G, [k][g][n Nb + m], and
    // lambda_x v(G)
    std::vector<zd> Mx;
    double vG[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double occ[4] = {0, 0, 0, 0};
    int c1 = 0;
};

void build_host_model(const tdagw_model_desc& d, HostModel& hm);

// ------------------------------------------------------------------ context ----------

// What the adjoint needs from the last checkpointed batched propagation.
struct AdjointState {
    bool valid = false;
    int B = 0, Bp = 0, Tmax = 0, period = 1, Rg = 0, Tg = 0, mode = 0;
    double dt = 0.0;
    std::vector<int> perm, steps;          // sorted -> caller order; caller-order lengths
    std::vector<tdagw_field> fields;       // caller order
    std::vector<unsigned char> fwd_args;   // argument block of the FP32 batched kernel
    const void* fwd_fn = nullptr;          // the FP32 forward kernel (for segment recomputes)
    // split-FP16 forward (tensor cores): its segment recomputes run the tensor-core kernel
    // (argument block, function, shared memory, CTAs); the backward sweep uses fwd_args
    bool tc = false;
    std::vector<unsigned char> tc_args;
    const void* tc_fn = nullptr;
    size_t tc_smem = 0;
    int tc_grid = 0;
};


// Channel-wise factors (Eq. svd-channel-wise), P = Nb^2 pairs.  Channel p -> q (output
// pair p, input pair q) has rank z[p P + q] (0 on the diagonal: diagonal channels are dense).
//   V segment q: Nk rows x ldv[q]; row k' = V^pq[k', 0:z_pq] for p != q, ascending p
//   U segment p: Nk rows x ldw[p]; row k  = U^pq[k, 0:z_pq] for q != p, ascending q
//                (nlr[p] columns), then K^pp[k, 0:Nk]
//   S, S o y, partials: sum_q ldv[q] entries aligned with the V columns (from sbase[q])
//   gidx: for each p (from gbase[p]), the S o y index of each low-rank column of its U rows
// Row lengths are even (a zero pad column) so every row starts on a 16-byte boundary.
constexpr int kMaxPairs = 16;
struct ChMeta {
    int P, Nk;
    int ldv[kMaxPairs], ldw[kMaxPairs], nlr[kMaxPairs];
    long long vbase[kMaxPairs], ubase[kMaxPairs], sbase[kMaxPairs], gbase[kMaxPairs];
    long long vtot, utot, stot, gtot;
};
struct ChannelFactors {
    bool valid = false;
    int zmax = 0;
    std::vector<int> z;     // P x P ranks
    std::vector<int> voff;  // [q P + p]: first column of channel p -> q in V segment q
    std::vector<int> uoff;  // [p P + q]: first column of channel p -> q in U segment p
    std::vector<int> gidx_host;
    ChMeta m{};
    DevBuf V, U, S, Y, gidx, part, Xt;
    // split-FP16 tiles of the segments for the tensor-core batched path, and whether they
    // match the installed factors
    bool tc_valid = false;
    DevBuf tcU, tcV, tcZero, tcGpad;
    float tc_su = 1.f, tc_sv = 1.f, tc_zbound = 0.f;
    std::vector<long long> tc_tvoff, tc_tuoff;
    std::vector<int> tc_mtq0, tc_nchw;
};

struct Ctx {
    tdagw_model_desc desc{};
    cudaStream_t stream = nullptr;
    HostModel hm;
    bool built = false;
    int dtype = TDAGW_C64;
    size_t csz = 8;  // bytes per complex element

    // model on device (context dtype)
    DevBuf K, diagK, dx, dy, vx, gap, Ud, Wd, Mxd, vGd;
    // low-rank factors K^off ~ U diag(S) V^H: U and V stored N x ldu row-major
    // (ldu = rank rounded up to even, zero pad column), S (rank, real of the dtype)
    DevBuf U, V, S, diagF;
    int rank = 0;
    // reading of K^diag in the low-rank form: 0 the strict diagonal (diagF), 1 the k = k'
    // blocks (kblkF: Nk x P x P, block k row p column q at (k P + p) P + q, P = Nb^2)
    int kdiag = 0;
    DevBuf kblkF;
    ChannelFactors ch;
    // propagation state (trajectory 0): compensated sum (Ssum + Ccomp), stage input X,
    // RK4 accumulator, dSigma, low-rank partials and projected vector
    DevBuf Ssum, Ccomp, X, acc, dS, ypart, ytil;
    DevBuf Etab, obs, red, counter, stepctr;
    int64_t step = 0;        // steps completed since the last reset
    int64_t obs_rows = 0;    // rows recorded by the last propagate
    int ysplit = 1;          // number of partial sums of V^H x

    // persistent low-rank launch: partial vectors, grid-barrier words and error flag
    DevBuf pbuf, sync;
    bool persistent_launched = false;
    // batched propagation: states N x Bp, intermediates, per-trajectory tables
    DevBuf bX, bS, bC, bA, bdS, bP, bY, bred, bobs, bEtab, bdir, bact, bperm, bfield, bchm;
    // (mode << 56 | B << 32 | rank) -> (row groups, traj groups); B <= 65536, rank < 2^32
    std::map<uint64_t, std::pair<int, int>> batch_plans;
    int last_plan_rg = 0, last_plan_tg = 0;
    int obs_B = 1;           // trajectories in the recorded observables
    // split-FP16 tiled factors for the tensor-core batched path, its intermediates, and
    // whether the tiles match the installed factors
    DevBuf tcU, tcV, tcY, tcP, tcMax, tcRed, tcDone, tcXt;
    bool tc_valid = false;
    float tc_su = 1.f, tc_sv = 1.f, tc_ybound = 0.f;
    // checkpoints (compensated state every `period` steps) and adjoint work buffers
    DevBuf ckS, ckC, aLam, aMu, aMusum, aC1, aMm, aKhm, aRecX, aRecDS;
    AdjointState adj;
    // stream used only to capture CUDA graphs (the caller's stream may be the legacy
    // default stream, on which capture is not allowed); graphs are launched on `stream`
    cudaStream_t cap = nullptr;
    // CUDA graphs of the batched launches (state resets + the persistent kernel), keyed by
    // the exact launch parameters and argument bytes; a few most recent kept
    struct BatchGraph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<BatchGraph> batch_graphs;
    bool batch_graphs_off = false;  // capture failed once on this device: launch directly
    ~Ctx() {
        for (BatchGraph& g : batch_graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (cap) cudaStreamDestroy(cap);
    }
};

// Row blocks of the stage-wise V^H x pass (each yields one partial vector): two per SM,
// at least 16 rows each.
inline int choose_ysplit(int r, int64_t N) {
    (void)r;
    int64_t nb = (N + 15) / 16;
    nb = nb < 304 ? nb : 304;
    return nb < 1 ? 1 : (int)nb;
}

// ------------------------------------------------------------------ launchers --------

template <typename R>
void launch_build_kernel(const Ctx& c, cudaStream_t s);
template <typename R>
void launch_gather_entries(const Ctx& c, const int64_t* rows, const int64_t* cols, int64_t n,
                           double2* out, cudaStream_t s);
// y[row] (+ diag[row] * xd[row]) = sum_j A[row, j] x[j] for rows [0, nrows); with nsplit > 1
// the columns are split and out holds nsplit partial vectors (no diag term then).
template <typename R>
void launch_gemv(const void* A, int64_t lda, int64_t nrows, int64_t ncols, const void* x,
                 void* out, int nsplit, const void* diag, const void* xd, cudaStream_t s);
// part[b][c] = sum over row block b of conj(V[i][c]) x_i, V stored N x ldv (rows)
template <typename R>
void launch_vcols(const void* V, int64_t ldv, int64_t N, int r, const void* x, void* part,
                  int nblocks, cudaStream_t s);
template <typename R>
void launch_yreduce(const void* part, int nsplit, int r, const void* S, void* ytil,
                    cudaStream_t s);
template <typename R>
void launch_stage(Ctx& c, int stage, double dt, double dirx, double diry, bool kahan,
                  cudaStream_t s);
template <typename R>
void launch_observables_row(Ctx& c, const void* X, int64_t row, cudaStream_t s);
void launch_field_table(const tdagw_field& f, double t_start, double dt, int64_t nsamp,
                        double* out, cudaStream_t s);
// analytic pulse parameters of one trajectory for the batched field tables
struct FieldParams {
    double E0, omega, t0, sigma, Tp;
    int kind;
    int64_t nsamp;
};
void launch_field_tables(const FieldParams* p_dev, int B, int64_t max_nsamp, int64_t ldE, double dt,
                         double* out, cudaStream_t s);
template <typename R>
void launch_convert_in(const double2* src, void* dst, int64_t n, cudaStream_t s);
template <typename R>
void launch_convert_out(const void* src, double2* dst, int64_t n, cudaStream_t s);

// Batched propagation of B trajectories (complex64, from drho = 0).
void propagate_batched(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt,
                       int mode, int flags);
// The same for the low-rank kernel with split-FP16 factors on the tensor cores.
void propagate_batched_tc(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt,
                          int flags);
// Split-FP16 tiled copies of the installed factors (made once per set of factors).
void pack_factors_tc(Ctx& c);
// The channel-wise kernel with split-FP16 segment tiles on the tensor cores.
void propagate_channel_tc(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt, int flags);

// One persistent cooperative launch of a batched kernel (argument block `args` of
// `args_size` bytes, a single by-value struct) after zeroing `resets` (pointer, bytes); with
// use_graph the sequence is replayed from a CUDA graph cached on the context.
struct ResetOp {
    void* p;
    size_t bytes;
};
void launch_batched(Ctx& c, const void* fn, dim3 grid, dim3 block, size_t smem, const void* args,
                    size_t args_size, const std::vector<ResetOp>& resets, bool use_graph);

// Host-side preparation shared by the batched drivers: trajectories sorted by length
// (longest first), active counts per step, per-trajectory field tables and directions,
// state buffers, and row 0 of the observables for every trajectory.
struct BatchSetup {
    std::vector<int> perm, act;
    int Tmax = 0, Bp = 0;
    int64_t ldE = 0, rows = 0;
};
BatchSetup prepare_batch(Ctx& c, const tdagw_field* fields, int B, const int* steps, double dt);
void reset_batch_observables(Ctx& c, const BatchSetup& bs, int B);
// observables in the caller's trajectory order
void finish_batch(Ctx& c, const BatchSetup& bs, int B);

// Backward sweep of the last checkpointed batched propagation (host arrays).
void adjoint_batched(Ctx& c, const double* dJdobs, double* dJdE, double* dJdparams);
// After a checkpointed tensor-core forward: the FP32 batched partition, launch arguments
// and intermediates of the adjoint's backward sweep, recorded in c.adj.
void prepare_adjoint_fp32(Ctx& c, const BatchSetup& bs, const tdagw_field* fields, int B, const int* steps,
                          double dt, int flags);
// Recompute steps [n0, n0 + len) of the last checkpointed tensor-core forward from the
// restored state (c.bS, c.bC, c.bX), recording every stage's input and dSigma.
void tc_recompute_segment(Ctx& c, int n0, int len, float2* recX, float2* recDS, double* obs);

// Persistent single-trajectory low-rank propagation (complex64); false if not applicable.
bool launch_lr_persistent(Ctx& c, int T, double dt, double dirx, double diry, bool kahan,
                          bool test_timeout, cudaStream_t s);

template <typename R>
void rsvd_compress(Ctx& c, int rank, int oversample, int power_iters, uint64_t seed);

// ---- channel-wise factors (channel.cu, rsvd.cu, ch_persistent.cu)
// Offsets and row lengths of the channel layout for ranks z (P x P); allocates and zeroes
// the factor arrays in the context dtype.
void ch_layout(Ctx& c, const std::vector<int>& z);
// dst[k ld + k'] = K[(k P + p) N + k' P + q] for the Nk x Nk channel p -> q (context dtype)
template <typename R>
void launch_ch_gather(const Ctx& c, int p, int q, void* dst, int64_t ld, cudaStream_t s);
// dst[k ld + off + j] = src[k z + j] (FP64 Nk x z into a segment of the context dtype)
template <typename R>
void launch_ch_place(const double2* src, int Nk, int z, void* dst, int64_t ld, int off,
                     cudaStream_t s);
// the dense diagonal channels of the built kernel into the U segments
template <typename R>
void ch_fill_diag_from_kernel(Ctx& c);
template <typename R>
void set_channel_factors(Ctx& c, int rank, const int* ranks, const double* U, const double* S,
                         const double* V, const double* D);
template <typename R>
void get_channel_factors(Ctx& c, int* rank, int* ranks, double* U, double* S, double* V,
                         double* D);
// y = K~ x with the channel-wise factors (stage-wise kernels)
template <typename R>
void launch_ch_apply(Ctx& c, const void* x, void* y, cudaStream_t s);
template <typename R>
void rsvd_channels(Ctx& c, int rank, int oversample, int power_iters, uint64_t seed,
                   double rel_tol);
// the k = k' blocks of the built kernel into dst (Nk x P x P, context dtype)
template <typename R>
void launch_gather_kblocks(const Ctx& c, void* dst, cudaStream_t s);
// y[k P + p] += sum_q B[k][p][q] x[k P + q] (context dtype; y may not alias x)
template <typename R>
void launch_kblock_add(const void* B, const void* x, void* y, int Nk, int P, cudaStream_t s);
// High-harmonic spectra of B recorded currents (host arrays in and out; synchronises).
void hhg_spectrum(const double* J, int64_t rows, int64_t stride, int B, const int* steps, double dt,
                  const double* omega, int nfreq, double* out, cudaStream_t s);
// Persistent single-trajectory channel-wise propagation (complex64); false if not applicable.
bool launch_ch_persistent(Ctx& c, int T, double dt, double dirx, double diry, bool kahan,
                          bool test_timeout, cudaStream_t s);

}  // namespace tdagw
