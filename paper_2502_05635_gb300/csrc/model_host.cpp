// Host-side (FP64) construction of the lattice model: analytic eigenpairs of each 2x2
// copy, band sorting, finite-difference Berry-connection dipoles, velocity, and the
// screened interaction W on grid offsets with its q = 0 mini-cell average.
//
// These are the k-local inputs of Eq. tdagw (H^QP diagonal in the band basis, the dipole
// matrix r of Appendix A.1) and of the direct kernel (Eq. bse-direct-def, with Bloch
// overlaps in place of plane-wave matrix elements and W(q=0) averaged over a small region
// as in Appendix B).  O(Nk) work; the O(N^2) kernel itself is written on the device.
#include <algorithm>
#include <array>
#include <cmath>

#include "common.cuh"

namespace tdagw {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Eig {
    int nb = 0, norb = 0;
    std::array<double, 4> e{};
    std::array<std::array<zd, 4>, 4> u{};  // u[n][orbital]
};

// Eigenpairs of the block-diagonal orbital Hamiltonian at (kx, ky) (1/bohr), sorted by
// energy.  For one block h = d.sigma + off:  E = off -+ |d|,
//   upper: (|d| + dz, dx + i dy) / sqrt(2|d|(|d| + dz)),
//   lower: (-(dx - i dy), |d| + dz) / sqrt(2|d|(|d| + dz)),
// valid while |d| + dz > 0 (dz >= Delta > 0 for this model).  The component |d| + dz is
// the larger in modulus and is real and positive: the gauge rule holds by construction.
Eig eigen(const tdagw_model_desc& p, double kx, double ky) {
    const double ca = kx * p.a, cb = ky * p.a;
    const double hx = p.t * std::sin(ca), hy = p.t * std::sin(cb);
    const double hz = p.Delta + p.m * (2.0 - std::cos(ca) - std::cos(cb));
    const double dn = std::sqrt(hx * hx + hy * hy + hz * hz);
    const double nrm = 1.0 / std::sqrt(2.0 * dn * (dn + hz));
    struct Cand { double e; int copy, upper; };
    std::vector<Cand> cs;
    for (int c = 0; c < p.nb_copies; ++c) {
        cs.push_back({p.offsets[c] - dn, c, 0});
        cs.push_back({p.offsets[c] + dn, c, 1});
    }
    std::stable_sort(cs.begin(), cs.end(), [](const Cand& a, const Cand& b) { return a.e < b.e; });
    Eig r;
    r.nb = r.norb = 2 * p.nb_copies;
    for (int n = 0; n < r.nb; ++n) {
        r.e[n] = cs[n].e;
        for (int o = 0; o < r.norb; ++o) r.u[n][o] = 0.0;
        const int o0 = 2 * cs[n].copy;
        if (cs[n].upper) {
            r.u[n][o0] = zd((dn + hz) * nrm, 0.0);
            r.u[n][o0 + 1] = zd(hx * nrm, hy * nrm);
        } else {
            r.u[n][o0] = zd(-hx * nrm, hy * nrm);
            r.u[n][o0 + 1] = zd((dn + hz) * nrm, 0.0);
        }
    }
    return r;
}

// dh/dk along `axis` for one block: a (t cos(k a) sigma_axis + m sin(k a) sigma_z)
void dh_block(const tdagw_model_desc& p, double kx, double ky, int axis, zd out[2][2]) {
    const double ka = (axis == 0 ? kx : ky) * p.a;
    const double c = p.a * p.t * std::cos(ka), z = p.a * p.m * std::sin(ka);
    out[0][0] = z;
    out[1][1] = -z;
    if (axis == 0) {
        out[0][1] = c;
        out[1][0] = c;
    } else {
        out[0][1] = zd(0.0, -c);
        out[1][0] = zd(0.0, c);
    }
}

zd inner(const std::array<zd, 4>& a, const std::array<zd, 4>& b, int norb) {
    zd s = 0.0;
    for (int o = 0; o < norb; ++o) s += std::conj(a[o]) * b[o];
    return s;
}

// Berry connection A_nm = i <u_n(k)| (u_m(k+d) - u_m(k-d)) / (2 d) > with each shifted
// u_m phase-aligned to u_m(k), Hermitised, diagonal zero (parallel-transport condition).
void berry(const tdagw_model_desc& p, double kx, double ky, int axis, const Eig& e0, zd* A) {
    const double del = 1e-5 / p.a;
    const double sx = axis == 0 ? del : 0.0, sy = axis == 1 ? del : 0.0;
    Eig ep = eigen(p, kx + sx, ky + sy), em = eigen(p, kx - sx, ky - sy);
    const int nb = e0.nb, no = e0.norb;
    for (int m = 0; m < nb; ++m) {
        zd op = inner(e0.u[m], ep.u[m], no), om = inner(e0.u[m], em.u[m], no);
        zd fp = std::conj(op) / std::abs(op), fm = std::conj(om) / std::abs(om);
        for (int o = 0; o < no; ++o) {
            ep.u[m][o] *= fp;
            em.u[m][o] *= fm;
        }
    }
    zd raw[4][4];
    for (int n = 0; n < nb; ++n)
        for (int m = 0; m < nb; ++m) {
            zd s = 0.0;
            for (int o = 0; o < no; ++o)
                s += std::conj(e0.u[n][o]) * (ep.u[m][o] - em.u[m][o]);
            raw[n][m] = zd(0.0, 1.0) * s / (2.0 * del);
        }
    for (int n = 0; n < nb; ++n)
        for (int m = 0; m < nb; ++m)
            A[n * nb + m] = (n == m) ? zd(0.0, 0.0) : 0.5 * (raw[n][m] + std::conj(raw[m][n]));
}

// Mean of W(q) = 2 pi / (A q (1 + r0 q)) over the square |qx|,|qy| <= h.  Splitting the
// square into 8 right triangles about the origin and integrating q W(q) radially in closed
// form, (2 pi / (A r0)) ln(1 + r0 h / cos th), leaves a smooth integral over th in
// [0, pi/4], evaluated here with composite Simpson on 4096 panels.
double mini_cell_average(double h, double A, double r0) {
    const int n = 4096;
    const double hstep = (kPi / 4.0) / n;
    auto f = [&](double th) { return std::log1p(r0 * h / std::cos(th)) / r0; };
    double s = f(0.0) + f(kPi / 4.0);
    for (int i = 1; i < n; ++i) s += (i % 2 ? 4.0 : 2.0) * f(i * hstep);
    const double ang = s * hstep / 3.0;
    return 8.0 * (2.0 * kPi / A) * ang / (4.0 * h * h);
}

}  // namespace

void build_host_model(const tdagw_model_desc& d, HostModel& hm) {
    const int L = d.L, nb = 2 * d.nb_copies, Nk = L * L;
    hm.L = L;
    hm.Nb = nb;
    hm.norb = nb;
    hm.Nk = Nk;
    hm.N = (int64_t)nb * nb * Nk;
    hm.eps.assign((size_t)Nk * nb, 0.0);
    hm.U.assign((size_t)Nk * nb * nb, 0.0);
    hm.dx.assign((size_t)Nk * nb * nb, 0.0);
    hm.dy.assign((size_t)Nk * nb * nb, 0.0);
    hm.vx.assign((size_t)Nk * nb * nb, 0.0);
    const double g = 2.0 * kPi / (L * d.a);
    for (int k = 0; k < Nk; ++k) {
        const double kx = (k / L) * g, ky = (k % L) * g;
        const Eig e = eigen(d, kx, ky);
        for (int n = 0; n < nb; ++n) {
            hm.eps[(size_t)k * nb + n] = e.e[n];
            for (int o = 0; o < nb; ++o) hm.U[((size_t)k * nb + o) * nb + n] = e.u[n][o];
        }
        berry(d, kx, ky, 0, e, &hm.dx[(size_t)k * nb * nb]);
        berry(d, kx, ky, 1, e, &hm.dy[(size_t)k * nb * nb]);
        zd blk[2][2];
        dh_block(d, kx, ky, 0, blk);
        for (int n = 0; n < nb; ++n)
            for (int m = 0; m < nb; ++m) {
                zd s = 0.0;
                for (int c = 0; c < d.nb_copies; ++c)
                    for (int i = 0; i < 2; ++i)
                        for (int j = 0; j < 2; ++j)
                            s += std::conj(e.u[n][2 * c + i]) * blk[i][j] * e.u[m][2 * c + j];
                hm.vx[((size_t)k * nb + n) * nb + m] = s;
            }
    }
    const double A = (double)Nk * d.a * d.a;
    hm.W0 = mini_cell_average(kPi / (L * d.a), A, d.r0);
    hm.Wtab.assign((size_t)L * L, 0.0);
    for (int di = 0; di < L; ++di)
        for (int dj = 0; dj < L; ++dj) {
            const int wi = di >= (L + 1) / 2 ? di - L : di;  // minimum image
            const int wj = dj >= (L + 1) / 2 ? dj - L : dj;
            const double q = std::hypot(wi * g, wj * g);
            hm.Wtab[(size_t)di * L + dj] =
                (di == 0 && dj == 0) ? hm.W0 : 2.0 * kPi / (A * q * (1.0 + d.r0 * q));
        }
    // exchange: point orbitals, orbital o at (o mod 2)(a/2, a/2), so exp(i G . tau_o) =
    // (-1)^((i + j)(o mod 2)) for G = (2 pi / a)(i, j)
    hm.Mx.clear();
    if (d.exchange > 0.0) {
        hm.Mx.assign((size_t)Nk * 8 * nb * nb, 0.0);
        int g = 0;
        for (int i = -1; i <= 1; ++i)
            for (int j = -1; j <= 1; ++j) {
                if (i == 0 && j == 0) continue;
                const double G = 2.0 * kPi / d.a * std::hypot((double)i, (double)j);
                hm.vG[g] = d.exchange * 2.0 * kPi / (A * G);
                const double odd = ((i + j) % 2 != 0) ? -1.0 : 1.0;
                for (int k = 0; k < Nk; ++k)
                    for (int n = 0; n < nb; ++n)
                        for (int m = 0; m < nb; ++m) {
                            zd s = 0.0;
                            for (int o = 0; o < nb; ++o) {
                                const double ph = (o % 2) ? odd : 1.0;
                                s += std::conj(hm.U[((size_t)k * nb + o) * nb + n]) * hm.U[((size_t)k * nb + o) * nb + m] * ph;
                            }
                            hm.Mx[(((size_t)k * 8 + g) * nb + n) * nb + m] = s;
                        }
                ++g;
            }
    }
    for (int n = 0; n < 4; ++n) hm.occ[n] = n < nb / 2 ? 1.0 : 0.0;
    hm.c1 = nb / 2;
}

}  // namespace tdagw
