// Host-side linear stability gate of libplbm (von Neumann analysis).
//
// A Fourier mode exp(i k.x) of a small perturbation of the uniform state
// f^eq(1, u, theta0) advances by A(k) = J S(k): S(k) = diag(exp(-i k.v_p)) is the
// pull f_in,p(x) = f_p(x - v_p) and J is the Jacobian of the BGK collision of
// Eq. (eq:srt) with the equilibrium of Eq. (eq:rdr).  The lattice is linearly
// stable at that state when every eigenvalue of every A(k) lies in |lambda| <= 1.
//
// J is exact to rounding: each column is the imaginary part of the collision of
// f^eq + i h e_p divided by h (complex-step derivative, h = 1e-30).  Eigenvalues
// come from a reduction to upper Hessenberg form by Householder reflections and
// shifted QR sweeps with Givens rotations and Wilkinson shifts (textbook
// eigenvalue-only algorithm on a complex matrix).
#include "plbm.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <thread>
#include <vector>

#include "plbm_internal.h"

namespace {

using cplx = std::complex<double>;

// Moments, equilibrium and BGK collision of one node, templated on the number
// type so that the complex step carries the derivative.
template <typename T>
void collide_node(int dim, int q1, const int* v, const double* C, double omega, double theta0,
                  bool isothermal, const T* fin, T* fout) {
    const int q = dim == 1 ? q1 : q1 * q1;
    T rho = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
    for (int p = 0; p < q; ++p) {
        const int ix = dim == 1 ? p : p / q1;
        const int iy = dim == 1 ? 0 : p % q1;
        const double vx = v[ix], vy = dim == 1 ? 0.0 : (double)v[iy];
        rho += fin[p];
        jx += vx * fin[p];
        jy += vy * fin[p];
        e += (vx * vx + vy * vy) * fin[p];
    }
    const T ux = jx / rho, uy = jy / rho;
    T th = (e / rho - (ux * ux + uy * uy)) / (double)dim;
    if (isothermal) th = theta0;
    T r[2][plbm::kMaxQ1];
    for (int a = 0; a < dim; ++a) {
        const T u = a == 0 ? ux : uy;
        T mu[plbm::kMaxQ1];
        mu[0] = 1.0;
        if (q1 > 1) mu[1] = u;
        for (int n = 1; n + 1 < q1; ++n) mu[n + 1] = u * mu[n] + (double)n * th * mu[n - 1];
        for (int i = 0; i < q1; ++i) {
            T s = 0.0;
            for (int n = 0; n < q1; ++n) s += C[i * q1 + n] * mu[n];
            r[a][i] = s;
        }
    }
    for (int p = 0; p < q; ++p) {
        const int ix = dim == 1 ? p : p / q1;
        const int iy = dim == 1 ? 0 : p % q1;
        const T feq = dim == 1 ? rho * r[0][ix] : rho * r[0][ix] * r[1][iy];
        fout[p] = (1.0 - omega) * fin[p] + omega * feq;
    }
}

// Eigenvalues of a complex n x n matrix (row-major, destroyed).
void eigenvalues(int n, std::vector<cplx>& A, std::vector<cplx>& lam) {
    auto at = [&](int i, int j) -> cplx& { return A[(size_t)i * n + j]; };
    // Balancing: a diagonal similarity D^-1 A D with powers of two that brings
    // the off-diagonal norm of each row close to that of its column.  The
    // collision Jacobian couples populations whose weights differ by more than
    // two orders of magnitude; balancing keeps the backward error of the QR
    // sweeps small relative to each entry, which matters for the nearly
    // defective eigenvalue clusters near |lambda| = 1.
    for (bool changed = true; changed;) {
        changed = false;
        for (int i = 0; i < n; ++i) {
            double c = 0.0, r = 0.0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                c += std::abs(at(j, i));
                r += std::abs(at(i, j));
            }
            if (c == 0.0 || r == 0.0) continue;
            double f = 1.0;
            const double s = c + r;
            double cc = c, rr = r;
            while (cc < rr / 2.0) {
                cc *= 2.0;
                rr /= 2.0;
                f *= 2.0;
            }
            while (cc >= rr * 2.0) {
                cc /= 2.0;
                rr *= 2.0;
                f /= 2.0;
            }
            if ((cc + rr) < 0.95 * s) {
                changed = true;
                for (int j = 0; j < n; ++j) at(i, j) /= f;
                for (int j = 0; j < n; ++j) at(j, i) *= f;
            }
        }
    }
    // Householder reduction to upper Hessenberg form.
    for (int k = 0; k + 2 < n; ++k) {
        double alpha2 = 0.0;
        for (int i = k + 1; i < n; ++i) alpha2 += std::norm(at(i, k));
        const double alpha = std::sqrt(alpha2);
        if (alpha == 0.0) continue;
        const cplx x0 = at(k + 1, k);
        const cplx phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cplx(1.0, 0.0);
        std::vector<cplx> w(n, 0.0);
        w[k + 1] = x0 + phase * alpha;
        for (int i = k + 2; i < n; ++i) w[i] = at(i, k);
        double wn = 0.0;
        for (int i = k + 1; i < n; ++i) wn += std::norm(w[i]);
        if (wn == 0.0) continue;
        // A <- (I - 2 w w^H / |w|^2) A (I - 2 w w^H / |w|^2)
        for (int j = 0; j < n; ++j) {
            cplx s = 0.0;
            for (int i = k + 1; i < n; ++i) s += std::conj(w[i]) * at(i, j);
            s *= 2.0 / wn;
            for (int i = k + 1; i < n; ++i) at(i, j) -= w[i] * s;
        }
        for (int i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int j = k + 1; j < n; ++j) s += at(i, j) * w[j];
            s *= 2.0 / wn;
            for (int j = k + 1; j < n; ++j) at(i, j) -= s * std::conj(w[j]);
        }
        for (int i = k + 2; i < n; ++i) at(i, k) = 0.0;
    }
    // Shifted QR on the active window [lo, hi].
    lam.assign(n, 0.0);
    int hi = n - 1;
    int iter = 0;
    const double eps = 2.2e-16;
    std::vector<cplx> cs(n), sn(n);
    while (hi >= 0) {
        if (hi == 0) {
            lam[0] = at(0, 0);
            break;
        }
        int lo = hi;
        while (lo > 0) {
            const double sc = std::abs(at(lo, lo)) + std::abs(at(lo - 1, lo - 1));
            if (std::abs(at(lo, lo - 1)) <= eps * (sc > 0.0 ? sc : 1.0)) {
                at(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            lam[hi] = at(hi, hi);
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 1000) {  // no convergence: report the diagonal (never seen in practice)
            for (int i = 0; i <= hi; ++i) lam[i] = at(i, i);
            break;
        }
        // Wilkinson shift from the trailing 2 x 2 block of the window.
        const cplx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
        const cplx tr = a + d, det = a * d - b * c;
        const cplx disc = std::sqrt(tr * tr / 4.0 - det);
        cplx m1 = tr / 2.0 + disc, m2 = tr / 2.0 - disc;
        cplx mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        if (iter % 11 == 10) mu = d + std::abs(at(hi, hi - 1)) * 0.75;  // exceptional shift
        // H - mu I = Q R with Givens rotations on the subdiagonal, then R Q + mu I.
        for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
        for (int k = lo; k < hi; ++k) {
            const cplx x = at(k, k), y = at(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            cplx ck, sk;
            if (r == 0.0) {
                ck = 1.0;
                sk = 0.0;
            } else {
                ck = x / r;
                sk = y / r;
            }
            cs[k] = ck;
            sn[k] = sk;
            for (int j = k; j <= hi; ++j) {
                const cplx t1 = at(k, j), t2 = at(k + 1, j);
                at(k, j) = std::conj(ck) * t1 + std::conj(sk) * t2;
                at(k + 1, j) = -sk * t1 + ck * t2;
            }
        }
        for (int k = lo; k < hi; ++k) {
            const cplx ck = cs[k], sk = sn[k];
            for (int i = lo; i <= std::min(k + 2, hi); ++i) {
                const cplx t1 = at(i, k), t2 = at(i, k + 1);
                at(i, k) = t1 * ck + t2 * sk;
                at(i, k + 1) = -t1 * std::conj(sk) + t2 * std::conj(ck);
            }
        }
        for (int i = lo; i <= hi; ++i) at(i, i) += mu;
    }
}

}  // namespace

namespace plbm {

double spectral_radius(int dim, int q1, const int* v, const double* C, double omega, double theta0,
                       bool isothermal, double ux, int nk, double stop_above) {
    const int q = dim == 1 ? q1 : q1 * q1;
    // f^eq(1, (ux, 0), theta0) from the rule, then the complex-step Jacobian of the collision.
    std::vector<cplx> f0(q), fo(q);
    {
        double r[2][kMaxQ1];
        for (int a = 0; a < dim; ++a) {
            const double u = a == 0 ? ux : 0.0;
            double mu[kMaxQ1];
            mu[0] = 1.0;
            if (q1 > 1) mu[1] = u;
            for (int n = 1; n + 1 < q1; ++n) mu[n + 1] = u * mu[n] + n * theta0 * mu[n - 1];
            for (int i = 0; i < q1; ++i) {
                double s = 0.0;
                for (int n = 0; n < q1; ++n) s += C[i * q1 + n] * mu[n];
                r[a][i] = s;
            }
        }
        for (int p = 0; p < q; ++p) {
            const int ix = dim == 1 ? p : p / q1;
            const int iy = dim == 1 ? 0 : p % q1;
            f0[p] = dim == 1 ? r[0][ix] : r[0][ix] * r[1][iy];
        }
    }
    const double h = 1e-30;
    std::vector<double> J((size_t)q * q);
    for (int p = 0; p < q; ++p) {
        std::vector<cplx> fin = f0;
        fin[p] += cplx(0.0, h);
        collide_node<cplx>(dim, q1, v, C, omega, theta0, isothermal, fin.data(), fo.data());
        for (int i = 0; i < q; ++i) J[(size_t)i * q + p] = fo[i].imag() / h;
    }
    // k-grid: kx in [0, pi] (A(-k) is the complex conjugate of A(k)); ky over the full
    // circle, or over [0, pi] when the set is symmetric (the state (ux, 0) is then
    // mirror-symmetric in y, and A(kx, -ky) is similar to A(kx, ky)).
    bool symmetric = true;
    for (int i = 0; i < q1 && symmetric; ++i) {
        bool found = false;
        for (int j = 0; j < q1; ++j) found |= (v[j] == -v[i]);
        symmetric = found;
    }
    std::vector<std::pair<double, double>> ks;
    const int nb = dim == 2 ? (symmetric ? nk / 2 + 1 : nk) : 1;
    for (int a = 0; a <= nk / 2; ++a)
        for (int b = 0; b < nb; ++b) ks.emplace_back(2.0 * M_PI * a / nk, 2.0 * M_PI * b / nk);
    // The narrowest unstable bands of tensor-product lattices lie on the axes
    // (modes that vary along one direction only): scan both axes 8x more densely.
    const int na = 8 * nk;
    for (int a = 1; a <= na / 2; ++a) {
        if (a % 8) ks.emplace_back(2.0 * M_PI * a / na, 0.0);
    }
    if (dim == 2) {
        const int nby = symmetric ? na / 2 : na - 1;
        for (int b = 1; b <= nby; ++b)
            if (b % 8) ks.emplace_back(0.0, 2.0 * M_PI * b / na);
    }
    std::vector<double> best(ks.size(), 0.0);
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::atomic<bool> stop{false};
    auto work = [&](unsigned t) {
        std::vector<cplx> A((size_t)q * q), lam;
        for (size_t k = t; k < ks.size() && !stop.load(std::memory_order_relaxed); k += hw) {
            for (int i = 0; i < q; ++i)
                for (int p = 0; p < q; ++p) {
                    const int ix = dim == 1 ? p : p / q1;
                    const int iy = dim == 1 ? 0 : p % q1;
                    const double ph = ks[k].first * v[ix] + (dim == 2 ? ks[k].second * v[iy] : 0.0);
                    A[(size_t)i * q + p] = J[(size_t)i * q + p] * std::exp(cplx(0.0, -ph));
                }
            eigenvalues(q, A, lam);
            double m = 0.0;
            for (const cplx& l : lam) m = std::max(m, std::abs(l));
            best[k] = m;
            if (stop_above > 0.0 && m > stop_above) stop.store(true, std::memory_order_relaxed);
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < hw; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
    return *std::max_element(best.begin(), best.end());
}

}  // namespace plbm
