// Per-element RK4 stage update of Eq. tdagw, shared by the stage-wise kernel and the
// persistent low-rank kernel: commutator of one Nb x Nb block with warp shuffles, the
// classical RK4 combination, the compensated state update, and the observables.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace tdagw {

template <typename C> __device__ __forceinline__ C shfl(C v, int src) {
    return mk(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
template <typename C> __device__ __forceinline__ C shfl_xor(C v, int m) {
    return mk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

template <typename R> struct GapT { using type = double; };
template <> struct GapT<float> { using type = float2; };  // (hi, lo) split of eps_n - eps_m

__device__ __forceinline__ float2 gap_times(float2 g, float2 x) {
    // (hi + lo) x with both products rounded separately: the systematic rounding of the
    // band gap, which would accumulate as a phase error over many steps, is kept to FP64
    // level while each product has only a random FP32 rounding
    return make_float2(fmaf(g.x, x.x, g.y * x.x), fmaf(g.x, x.y, g.y * x.y));
}
__device__ __forceinline__ double2 gap_times(double g, double2 x) {
    return make_double2(g * x.x, g * x.y);
}

// error-free sum a + b = s + e (Knuth TwoSum)
template <typename R> __device__ __forceinline__ R two_sum(R a, R b, R& e) {
    const R s = a + b;
    const R bp = s - a;
    e = (a - (s - bp)) + (b - bp);
    return s;
}

template <typename R>
struct StageParams {
    using C = cplx_t<R>;
    const C* X;       // stage input X_s
    const C* dS;      // K . X_s
    const C* dx;
    const C* dy;
    const C* vx;
    const typename GapT<R>::type* gap;
    C* acc;           // k1 + 2 k2 + 2 k3 (+ k4)
    C* Ssum;          // state drho_n = Ssum + Ccomp
    C* Ccomp;
    C* Xnext;         // next stage input (may alias X: each element is read before written)
    const double* Etab;   // E at half-step times of this call
    int64_t* step;        // steps done in this call (device counter; stage-wise path)
    double* obs;          // (rows, 3)
    double* red;          // block partials of the observables
    unsigned* counter;    // arrival counter of the last-block reduction
    int64_t N;
    int Nk, c1;
    R occ[4];
    R dt, dirx, diry;
    int stage, kahan;
};

struct Obs3 {
    double p, j, o;
};

// Double-float sums (hi, lo) in FP32: error-free products (FMA) and sums (TwoSum), the
// compensated dot product of Ogita, Rump and Oishi (2005).  FP64 arithmetic is slow on this
// GPU; double-float keeps a few units of 2^-44 of the FP64 result and runs on FP32 pipes.
struct DF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float s = hi + v, bp = s - hi;
        lo += (hi - (s - bp)) + (v - bp);
        hi = s;
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        const float ep = fmaf(a, b, -p);
        add(p);
        lo += ep;
    }
    __device__ __forceinline__ void add(const DF& o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ DF shfl_xor_sum(int m) const {
        DF r = *this;
        DF t;
        t.hi = __shfl_xor_sync(0xffffffffu, hi, m);
        t.lo = __shfl_xor_sync(0xffffffffu, lo, m);
        r.add(t);
        return r;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
// observable sums of P_x, J_x and the occupation: FP64 (Obs3) or double-float (ObsDF)
struct ObsDF {
    DF p, j, o;
};
__device__ __forceinline__ void obs_add_prod(Obs3& ob, int w, double a, double b) {
    (w == 0 ? ob.p : ob.j) += a * b;
}
__device__ __forceinline__ void obs_add_prod(ObsDF& ob, int w, float a, float b) {
    (w == 0 ? ob.p : ob.j).add_prod(a, b);
}
__device__ __forceinline__ void obs_add_occ(Obs3& ob, double v) { ob.o += v; }
__device__ __forceinline__ void obs_add_occ(ObsDF& ob, float v) { ob.o.add(v); }

// Element i = (k Nb + n) Nb + m of stage `stage` at field amplitude E.  All NB^2 lanes of a
// k block must call this together (act = false for padding lanes).  Computes
//   k_s = -i [diag(eps) + E d + dSigma, rho0 + X_s]_nm
//       = -i ( (eps_n - eps_m) X_nm + M_nm (f_m - f_n) + sum_l (M_nl X_lm - X_nl M_lm) ),
// M = E d + dSigma, updates the RK4 accumulator and writes the next stage input; on the
// last stage advances the state (TwoSum compensation) and returns the element's share of
// Re Tr(rho d^x), Re Tr(rho v^x) and the first-conduction-band occupation, added to ob
// (FP64 sums: Obs3, double-float sums of FP32 values: ObsDF).
template <typename R, int NB, typename OB>
__device__ __forceinline__ void stage_element(const StageParams<R>& p, int64_t i, bool act,
                                              int lane, int stage, R E, OB& ob) {
    using C = cplx_t<R>;
    constexpr int NB2 = NB * NB;
    const int base = lane - (lane % NB2);
    const int g = lane % NB2, n = g / NB, m = g % NB;
    const C zero = mk((R)0, (R)0);
    // buffers rewritten during a launch are read through L2 only (ld.global.cg): a
    // persistent launch rereads them after other CTAs have stored new values
    const C X = act ? __ldcg(p.X + i) : zero;
    const C dS = act ? __ldcg(p.dS + i) : zero;
    const C dxv = act ? p.dx[i] : zero;
    const C dyv = act ? p.dy[i] : zero;
    const C M = cadd(dS, mk(E * (p.dirx * dxv.x + p.diry * dyv.x), E * (p.dirx * dxv.y + p.diry * dyv.y)));
    C comm = cscale(M, p.occ[m] - p.occ[n]);
#pragma unroll
    for (int l = 0; l < NB; ++l) {
        const C Mnl = shfl(M, base + n * NB + l);
        const C Xlm = shfl(X, base + l * NB + m);
        const C Xnl = shfl(X, base + n * NB + l);
        const C Mlm = shfl(M, base + l * NB + m);
        comm = cfma(Mnl, Xlm, comm);
        comm = csub(comm, cmul(Xnl, Mlm));
    }
    if (act) {
        const C h0 = gap_times(p.gap[i], X);
        const C s = cadd(h0, comm);
        const C kv = mk(s.y, -s.x);  // -i s
        const C xs = __ldcg(p.Ssum + i), xc = __ldcg(p.Ccomp + i);
        C Xn;
        if (stage < 3) {
            const C a = stage == 0 ? kv : cadd(__ldcg(p.acc + i), cscale(kv, (R)2));
            p.acc[i] = a;
            const R cn = stage == 2 ? p.dt : (R)0.5 * p.dt;
            Xn = cadd(xs, cadd(xc, cscale(kv, cn)));
        } else {
            const C a = cadd(__ldcg(p.acc + i), kv);
            const C inc = cscale(a, p.dt / (R)6);
            C ns, nc;
            if (p.kahan) {
                R ex, ey;
                ns.x = two_sum(xs.x, inc.x, ex);
                ns.y = two_sum(xs.y, inc.y, ey);
                nc = mk(xc.x + ex, xc.y + ey);
            } else {
                ns = cadd(xs, inc);
                nc = xc;
            }
            p.Ssum[i] = ns;
            p.Ccomp[i] = nc;
            Xn = cadd(ns, nc);
            // Re(rho_nm conj(d_nm)) summed over n, m is Re Tr(rho d) for Hermitian d
            const C rho = (n == m) ? cadd(Xn, mk(p.occ[n], (R)0)) : Xn;
            const C vxv = p.vx[i];
            using A = typename std::conditional<std::is_same<OB, Obs3>::value, double, float>::type;
            obs_add_prod(ob, 0, (A)rho.x, (A)dxv.x);
            obs_add_prod(ob, 0, (A)rho.y, (A)dxv.y);
            obs_add_prod(ob, 1, (A)rho.x, (A)vxv.x);
            obs_add_prod(ob, 1, (A)rho.y, (A)vxv.y);
            if (n == m && n == p.c1) obs_add_occ(ob, (A)rho.x);
        }
        p.Xnext[i] = Xn;
    }
}

}  // namespace tdagw
