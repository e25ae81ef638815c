/*
 * tdagw.h -- C ABI of the GB300 (sm_103a) TD-aGW kernel-contraction library.
 *
 * The library propagates the one-body density matrix of a crystal under a driving field,
 * Eq. tdagw of arXiv:2502.05635 ("Data-driven low-rank approximation for electron-hole
 * kernel and acceleration of time-dependent GW calculations"):
 *
 *     i d/dt rho_k = [ H^QP_k + dSigma_k(t) + E(t).d_k , rho_k ]
 *     dSigma_{nmk} = sum_{n'm'k'} K_{nmk,n'm'k'} drho_{n'm'k'}        (Eq. sigma-from-k)
 *
 * with the kernel applied either densely (cost Nb^4 Nk^2 per evaluation, Sec. "SVD
 * acceleration", Appendix A.1) or in the truncated-SVD form of Eq. svd_diag_offdiag /
 * Eq. svd_acc, dSigma = K^diag drho + U diag(S) (V^H drho) (cost Nb^2 Nk 2z).
 *
 * Conventions shared by every call
 *   - N = Nb^2 Nk; pair index i = (k Nb + n) Nb + m; k = ix L + iy on the L x L grid.
 *   - Complex numbers are interleaved (re, im).  "c64" = 2 x float, "c128" = 2 x double.
 *     The context's dtype (TDAGW_C64 or TDAGW_C128) fixes the device storage and the
 *     arithmetic of the propagation path; host-side exchange arrays are always c128/double.
 *   - Return value: TDAGW_OK (0) or a negative TDAGW_ERR_* code; tdagw_last_error() gives a
 *     message for the calling thread.  No C++ exception or abort crosses this boundary.
 *   - Device pointers passed in are borrowed for the duration of the call and used on the
 *     context's stream; all device work is stream-ordered on that stream.  Calls that write
 *     to host memory synchronise the stream before returning.
 *   - Memory the library allocates is owned by the context and freed by tdagw_destroy.
 */
#ifndef TDAGW_H
#define TDAGW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TDAGW_OK = 0,
    TDAGW_ERR_INVALID_ARG = -1,
    TDAGW_ERR_OOM = -2,
    TDAGW_ERR_CUDA = -3,
    TDAGW_ERR_NOT_BUILT = -4,     /* tdagw_build_kernel has not run */
    TDAGW_ERR_NO_FACTORS = -5,    /* low-rank mode without factors */
    TDAGW_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up */
    TDAGW_ERR_UNSUPPORTED = -7
};

enum { TDAGW_C64 = 0, TDAGW_C128 = 1 };
enum { TDAGW_FULL = 0, TDAGW_LOWRANK = 1, TDAGW_CHANNEL = 2 };
enum {
    TDAGW_FIELD_GAUSS_COS = 0,    /* E0 exp(-(t-t0)^2 / (2 sigma^2)) cos(omega t)          */
    TDAGW_FIELD_CONST = 1,        /* E0                                                     */
    TDAGW_FIELD_SIN2_SIN = 2,     /* E0 sin^2(pi t / T_pulse) sin(omega t) on [0, T_pulse]  */
    TDAGW_FIELD_TABLE = 3         /* caller samples E(j dt/2), j = 0 .. 2 steps              */
};
/* propagate flags */
enum {
    TDAGW_FLAG_RESET = 1,         /* start from drho = 0 and t = 0 (else continue)          */
    TDAGW_FLAG_NO_GRAPH = 2,      /* launch stage by stage instead of replaying a CUDA graph */
    TDAGW_FLAG_NO_KAHAN = 4,      /* plain (uncompensated) RK4 accumulation                 */
    TDAGW_FLAG_STAGEWISE = 8,     /* low-rank or channel-wise c64: stage-wise kernels
                                     instead of the persistent single-launch kernel         */
    TDAGW_FLAG_TEST_TIMEOUT = 16, /* fault-injection hook for tests: the grid barrier of the
                                     persistent single-trajectory kernels and of the
                                     batched kernels (no tuning runs then) waits
                                     for one block that does not exist,
                                     every wait runs out a 20 ms budget and the call ends
                                     with TDAGW_ERR_TIMEOUT at the next synchronising call   */
    TDAGW_FLAG_CHECKPOINT = 32,   /* keep checkpoints for tdagw_adjoint (runs the batched
                                     path, also for B = 1; needs TDAGW_FLAG_RESET)           */
    TDAGW_FLAG_SPLIT_F16 = 64     /* low-rank or channel-wise c64 (any B, needs
                                     TDAGW_FLAG_RESET): factors as
                                     split FP16 pairs (hi + lo) on the tensor cores with FP32
                                     accumulation (three products per term); with
                                     TDAGW_FLAG_CHECKPOINT the checkpointed run and the
                                     adjoint's segment recomputes run on the tensor cores    */
};

typedef struct tdagw_ctx tdagw_ctx;

/* Lattice stand-in for the paper's first-principles bands (Appendix A): nb_copies copies of
 * h(k) = Delta sz + t (sin(kx a) sx + sin(ky a) sy) + m (2 - cos kx a - cos ky a) sz,
 * copy c shifted by offsets[c]; Nb = 2 nb_copies bands, lower half occupied.  W(q) is the
 * 2D Rytova-Keldysh interaction 2 pi / (A |q| (1 + r0 |q|)), A = Nk a^2, with W(0) the
 * mean over the grid's mini-cell (Appendix B).  With exchange = lambda_x > 0 the kernel
 * also holds the exchange term of Eq. bse-exchange-def at Q = 0 for point orbitals (orbital
 * o of each copy at (o mod 2) (a/2, a/2)) and the eight reciprocal vectors
 * G = (2 pi / a)(i, j), |i|, |j| <= 1, G != 0:
 *   K^x_{(k n m),(k' n' m')} = lambda_x sum_G v(G) M_nm(k, G) conj(M_n'm'(k', G)),
 *   M_nm(k, G) = sum_o conj(U_k[o, n]) U_k[o, m] exp(i G . tau_o), v(G) = 2 pi / (A |G|). */
typedef struct {
    int L;                /* grid is L x L, 1 <= L <= 4096                                */
    int nb_copies;        /* 1 (Nb = 2) or 2 (Nb = 4)                                     */
    double offsets[4];    /* energy offset of each copy (Ha)                              */
    double Delta, t, m;   /* model parameters (Ha)                                        */
    double a;             /* lattice constant (bohr)                                      */
    double r0;            /* screening length (bohr)                                      */
    int dtype;            /* TDAGW_C64 or TDAGW_C128                                      */
    double exchange;      /* lambda_x >= 0: scale of the exchange term (0 = direct only)  */
} tdagw_model_desc;

/* One driving pulse (atomic units).  The field is E(t) (dir_x, dir_y) and couples as
 * E(t).d_k with the k-local dipoles d (Eq. tdagw, length gauge). */
typedef struct {
    int kind;             /* TDAGW_FIELD_*                                                */
    double E0, omega, t0, sigma, T_pulse;
    double dir_x, dir_y;
    const double* table;  /* kind TABLE: host array of 2*steps+1 samples, else NULL       */
} tdagw_field;

/* Create a context for one model.  stream: the cudaStream_t all work of this context is
 * ordered on (NULL = the legacy default stream; CUDA graphs are captured on a private
 * stream and launched on this one).  *out receives the context.  Allocates nothing on
 * the device yet. */
int tdagw_create(const tdagw_model_desc* desc, void* stream, tdagw_ctx** out);

/* Build the model (bands, gauge-fixed eigenvectors, dipoles d^x, d^y, velocity v^x) on the
 * host in FP64 and the dense kernel K (N x N, row-major, context dtype) on the device
 * (Eq. bse-direct-def for the model:
 *   K_{(k n m),(k' n' m')} = -W(k - k') (U_k^+ U_k')_{n n'} (U_k'^+ U_k)_{m' m}).
 * Errors: TDAGW_ERR_OOM if K does not fit. */
int tdagw_build_kernel(tdagw_ctx* ctx);

/* Sizes: N = Nb^2 Nk, Nb, Nk.  Any pointer may be NULL. */
int tdagw_model_info(const tdagw_ctx* ctx, int64_t* N, int* Nb, int* Nk);

/* Copy the host-side model out (for checks).  eps: Nk*Nb doubles; dx, dy, vx: Nk*Nb*Nb c128;
 * U: Nk*Norb*Nb c128 (column n of U_k is band n in the orbital basis).  Any may be NULL. */
int tdagw_get_model(const tdagw_ctx* ctx, double* eps, double* dx, double* dy, double* vx,
                    double* U);

/* Sampled kernel entries K[rows[i], cols[i]] as stored on the device, written to out as
 * n c128 values (host).  Synchronises. */
int tdagw_get_kernel_entries(tdagw_ctx* ctx, const int64_t* rows, const int64_t* cols,
                             int64_t n, double* out);

/* Randomised truncated SVD of K^off = K - diag(K) (Eq. svd_diag_offdiag) to rank `rank`
 * (Halko-Martinsson-Tropp range finder with `oversample` extra columns and `power_iters`
 * power iterations, Gaussian test matrix from `seed`; FP64 orthogonalisation and core
 * eigen-solve on the device, K^off being Hermitian).  Replaces any factors present.
 * precision: 0 = factors stored in the context dtype; 1 = in addition, the split-FP16
 * tiled copy used by TDAGW_FLAG_SPLIT_F16 is made now (otherwise on first use after the
 * factors change; complex64 contexts only).  Errors: INVALID_ARG if rank + oversample > N
 * or precision is not 0 or 1; UNSUPPORTED for precision 1 on a complex128 context. */
int tdagw_compress_svd(tdagw_ctx* ctx, int rank, int oversample, int power_iters,
                       uint64_t seed, int precision);

/* Reading of K^diag in the low-rank form (Sec. "SVD analysis": "n1, n2, k = n3, n4, k'"):
 * on = 0 (default) the strict matrix diagonal; on = 1 the k = k' blocks, Nb^2 x Nb^2 per
 * k-point, so K^off = K minus those blocks and dSigma_k = B_k drho_k + (U (S o (V^H drho)))_k.
 * Changing it removes installed low-rank factors (they split K the other way).  With on = 1,
 * tdagw_compress_svd factors K minus the blocks, and the diag argument of tdagw_set_factors /
 * tdagw_get_factors holds the blocks (Nk x P x P c128, block k row p column q at
 * (k P + p) P + q, P = Nb^2; NULL in set: the blocks of the built kernel).  Supported by
 * tdagw_apply, tdagw_propagate (single trajectory and batched FP32) and tdagw_adjoint;
 * split-FP16 factors return UNSUPPORTED while it is on.  Errors: INVALID_ARG for on not 0
 * or 1. */
int tdagw_set_kdiag_blocks(tdagw_ctx* ctx, int on);

/* Install factors K^off ~ U diag(S) V^H from the host (c128 U, V: N x rank row-major;
 * S: rank doubles; diag: N c128 or NULL to keep diag(K) of the built kernel; the k-block
 * form of tdagw_set_kdiag_blocks when that is on). */
int tdagw_set_factors(tdagw_ctx* ctx, int rank, const double* U, const double* S,
                      const double* V, const double* diag);

/* Copy the installed factors to the host in c128 (U, V: N x rank; S: rank; diag: N, or the
 * Nk x P x P blocks with the k-block reading of K^diag).  *rank receives the rank; any array
 * pointer may be NULL. */
int tdagw_get_factors(tdagw_ctx* ctx, int* rank, double* U, double* S, double* V, double* diag);

/* Channel-wise compression (Sec. "SVD analysis of electron-hole kernel", Eq.
 * svd-channel-wise).  With pair indices p = n1 Nb + n2 and q = n3 Nb + n4 (P = Nb^2 pairs),
 * channel p -> q is the Nk x Nk block K^pq[k, k'] = K[k P + p, k' P + q].  Diagonal channels
 * (p = q, close to full rank) are kept exact as dense blocks; every off-diagonal channel holds
 * its own truncated SVD K^pq ~ U^pq diag(S^pq) (V^pq)^H of rank z_pq (0 <= z_pq <= Nk).
 * Mode TDAGW_CHANNEL of tdagw_apply / tdagw_propagate applies
 *   dSigma[k P + p] = sum_k' K^pp[k, k'] x[k' P + p] + sum_{q != p} U^pq (S^pq o ((V^pq)^H x_q)),
 * x_q[k'] = x[k' P + q].  Channel factors are independent of the low-rank factors above.
 *
 * tdagw_compress_channels: randomised SVD of every off-diagonal channel p < q of the built
 * kernel (Gaussian range finder with `oversample` extra columns, at most Nk in all, and
 * `power_iters` power iterations, test matrices from `seed`; FP64 orthogonalisation; the
 * core from the eigen-decomposition of B B^H, B = Q^H K^pq), keeping of the `rank` largest
 * singular values those above rel_tol times the channel's largest (a vanishing channel gets
 * rank 0); channel q -> p is the conjugate transpose of p -> q (K is Hermitian).  Diagonal
 * channels are copied from the kernel.  Replaces any channel factors present.  Errors:
 * INVALID_ARG for rank outside [0, Nk], oversample < 0, power_iters < 0 or rel_tol < 0;
 * NOT_BUILT before tdagw_build_kernel. */
int tdagw_compress_channels(tdagw_ctx* ctx, int rank, int oversample, int power_iters,
                            uint64_t seed, double rel_tol);

/* Install channel factors from the host (c128 / double):
 *   ranks  P x P ints, z_pq at p P + q (diagonal entries ignored); NULL: every
 *          off-diagonal channel has rank `rank`.  0 <= z_pq <= rank <= Nk.
 *   U, V   P x P x Nk x rank: U^pq[k, j] at ((p P + q) Nk + k) rank + j (columns j >= z_pq
 *          and the diagonal channels are ignored); may be NULL when rank = 0.
 *   S      P x P x rank, S^pq[j] at (p P + q) rank + j.
 *   D      P x Nk x Nk, K^pp[k, k'] at (p Nk + k) Nk + k'; NULL: taken from the built kernel.
 * Errors: INVALID_ARG for ranks out of range or a NULL factor array with rank > 0;
 * NOT_BUILT before tdagw_build_kernel (the layout takes Nb and Nk from the built model). */
int tdagw_set_channel_factors(tdagw_ctx* ctx, int rank, const int* ranks, const double* U,
                              const double* S, const double* V, const double* D);

/* Copy the channel factors to the host in the layout of tdagw_set_channel_factors with
 * rank = the largest z_pq (*rank), zero beyond each channel's own rank (ranks: P x P,
 * 0 on the diagonal).  Any pointer may be NULL.  Synchronises.  Errors: NO_FACTORS if no
 * channel factors are installed and an array is requested. */
int tdagw_get_channel_factors(tdagw_ctx* ctx, int* rank, int* ranks, double* U, double* S,
                              double* V, double* D);

/* One kernel application y = K x (mode FULL), y = K^diag x + U (S (V^H x)) (LOWRANK) or the
 * channel-wise form above (CHANNEL) on device vectors of N elements in the context dtype. */
int tdagw_apply(tdagw_ctx* ctx, int mode, const void* x, void* y);

/* Propagate B trajectories by classical RK4 (four stages per step, dSigma re-evaluated at
 * every stage, Kahan-compensated state accumulation) for steps[b] steps of dt; trajectory b
 * is driven by fields[b] (B host structs).  Observables (P_x, J_x, occupation of the first
 * conduction band; Sec. "SVD acceleration") are recorded at every step including t = 0.
 * B = 1: the single-trajectory path (continues from the current state unless
 * TDAGW_FLAG_RESET).  B > 1 (complex64 contexts): all trajectories in one persistent
 * launch, each starting from drho = 0 (TDAGW_FLAG_RESET required); trajectories of
 * different lengths are sorted so finished ones stop costing work; the state buffers of
 * the single-trajectory path are not touched.
 * With TDAGW_FLAG_SPLIT_F16 (LOWRANK, complex64, any B) the two products of Eq. svd_acc run
 * on the tensor cores with the factors split into FP16 hi + lo pairs and FP32
 * accumulation; P(t) then agrees with the FP32 path to about 1e-6 relative.
 * Mode CHANNEL (channel-wise factors, Eq. svd-channel-wise) runs without
 * TDAGW_FLAG_CHECKPOINT; for B = 1 one persistent launch for complex64 when every input
 * pair's channels hold at most 2048 columns in all (else stage-wise kernels), for B > 1 the
 * batched FP32 launch; with TDAGW_FLAG_SPLIT_F16 (complex64, any B, TDAGW_FLAG_RESET) the
 * V segments and the U segments (low-rank columns and the dense diagonal channel of each
 * output pair) run on the tensor cores as split FP16 tiles, made at the first such call
 * after new channel factors.
 * Errors: NO_FACTORS for LOWRANK or CHANNEL without the matching factors; NOT_BUILT before
 * tdagw_build_kernel;
 * UNSUPPORTED for B > 1 on a complex128 context or without TDAGW_FLAG_RESET, and for
 * CHANNEL with TDAGW_FLAG_CHECKPOINT; INVALID_ARG for TDAGW_FLAG_SPLIT_F16 with FULL.
 * The work split of a tensor-core launch (trajectory groups of the U product, K-ranges of
 * V^H X, and per-tile counters or a grid barrier between a stage's epilogue and the next
 * V^H X; channel-wise: trajectory groups and K-ranges of the U segments) is tuned by
 * timing six steps of each candidate on the first call of at least eight steps for a
 * batch size and rank, and kept on the context. */
int tdagw_propagate(tdagw_ctx* ctx, const tdagw_field* fields, int B, const int* steps,
                    double dt, int mode, int flags);

/* Gradients through the last tdagw_propagate (run with TDAGW_FLAG_CHECKPOINT) by the exact
 * discrete adjoint of its RK4 steps.  The objective is any function of the recorded
 * observables; the caller passes its derivatives dJdobs (host, (max steps + 1) x B x 3,
 * the layout of tdagw_observables; entries after a trajectory's end are ignored).
 * Outputs (host, may be NULL): dJdE ((2 max steps + 1) x B): dJ/dE_j for the field sample
 * E(j dt/2) of each trajectory (the amplitude along its direction); dJdparams (B x 4):
 * dJ/d(E0, omega, t0, sigma) for TDAGW_FIELD_GAUSS_COS pulses (zeros otherwise).  The
 * backward sweep recomputes the forward run segment by segment from checkpoints taken
 * every ceil(sqrt(steps)) steps (on the tensor cores when the forward ran with
 * TDAGW_FLAG_SPLIT_F16; the reverse stages use the FP32 factors).  Synchronises.  Errors: INVALID_ARG without a
 * checkpointed run; UNSUPPORTED on complex128 contexts; TIMEOUT if a bounded wait gave up. */
int tdagw_adjoint(tdagw_ctx* ctx, const double* dJdobs, double* dJdE, double* dJdparams);

/* Copy the observables recorded by the last tdagw_propagate: rows (max steps + 1) x B x 3
 * FP64, row-major, trajectories in the caller's order; entries after a trajectory's last
 * step are NaN.  host != 0: out is host memory (synchronises); else device memory.
 * max_rows bounds the rows written; *rows receives the rows available. */
int tdagw_observables(tdagw_ctx* ctx, double* out, int64_t max_rows, int64_t* rows, int host);

/* State of trajectory 0: drho (N c128, host) = compensated sum + carry, the carry alone
 * (N c128, the low-order part kept by the compensated RK4 accumulation; may be NULL) and
 * the steps taken since the last reset.  set_state installs them (carry NULL = zero);
 * get_state followed by set_state resumes a run bit for bit.  Synchronises. */
int tdagw_get_state(tdagw_ctx* ctx, double* drho, double* carry, int64_t* step);
int tdagw_set_state(tdagw_ctx* ctx, const double* drho, const double* carry, int64_t step);

/* Allocation-free variant of the low-rank contraction (the paper has no counterpart: this
 * is a deployment convenience).  Computes y = diag o x + U (S o (V^H x)) like
 * tdagw_apply(TDAGW_LOWRANK), but on arrays the caller owns and without allocating any
 * device memory.  It is meant for callers that cannot call cudaMalloc on their call path:
 * code whose device memory belongs to another framework's pool (a direct allocation would
 * escape that pool's accounting and limits), loops that must not take the implicit device
 * synchronisation of cudaMalloc/cudaFree, and processes running at a hard memory cap.
 *
 *   U, V    device, complex64, N x ld row-major (rows 16-byte aligned: ld even), columns
 *           [0, rank) used; the factors of K^off ~ U diag(S) V^H.
 *   S       device, rank floats.
 *   diag    device, N complex64 (K^diag).
 *   x, y    device, N complex64 each, 16-byte aligned, not aliasing.
 *   stream  cudaStream_t the work is queued on (NULL = legacy default stream).
 *
 * Intermediate vectors live in one fixed device array of 2.4 MiB ((152 + 1) x 2048
 * complex64) defined in the library, which every GPU that loads the library holds until
 * the process exits; rank above 2048 is rejected with TDAGW_ERR_INVALID_ARG.  The first
 * call on each device looks up that array's device address (cudaGetSymbolAddress, which
 * may load the library's device code); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents; every value a call
 * reads from it is written by the same call first, so nothing needs clearing.  Calls
 * whose work overlaps on the GPU (other streams, other host threads) race on the array:
 * serialise them.  The work runs on the current device; every array must be device (or
 * managed) memory of that device.  Errors: TDAGW_ERR_INVALID_ARG for NULL or misaligned
 * pointers, N < 1, rank outside [1, 2048], odd ld or ld < rank, and for a pointer that is
 * host memory or memory of another device; TDAGW_ERR_CUDA if the address lookup or a
 * launch fails. */
int tdagw_apply_lowrank_noalloc(const void* U, const void* V, int64_t ld, const float* S,
                                const void* diag, int64_t N, int rank, const void* x, void* y,
                                void* stream);

/* High-harmonic spectra (Sec. "SVD acceleration of TD-aGW": HHG(w) = |w int J(t) e^{-i w t} dt|^2)
 * of B recorded currents, e.g. the J column of tdagw_observables after an angle or
 * frequency sweep (Appendix C).  Integral by the rectangle rule over t_n = n dt,
 * n = 0 .. steps[b].
 *   J       host doubles; J_b(t_n) at J[(n B + b) stride] (stride 3 and J = obs + 1 for the
 *           observables array of tdagw_observables, stride 1 for a plain rows x B array).
 *   rows    rows of J (at least max steps + 1).
 *   omega   host, nfreq angular frequencies;  out: host, nfreq x B, HHG_b(omega_f) at f B + b.
 *   stream  cudaStream_t the work is queued on (NULL = legacy default stream).
 * FP64 on the GPU; allocates and frees its device buffers; synchronises.  Errors:
 * INVALID_ARG for NULL pointers, B, nfreq, stride or rows < 1, B > 65535, dt <= 0, a
 * negative step count, or rows < max steps + 1. */
int tdagw_hhg_spectrum(const double* J, int64_t rows, int64_t stride, int B, const int* steps,
                       double dt, const double* omega, int nfreq, double* out, void* stream);

/* Wait for all work queued on the context's stream.  Reports TDAGW_ERR_TIMEOUT if a bounded
 * device-side wait of the last propagation gave up (also reported by tdagw_observables to
 * host memory and tdagw_get_state). */
int tdagw_sync(tdagw_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* tdagw_last_error(void);

void tdagw_destroy(tdagw_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TDAGW_H */
