// Plan-time least-misfit gridding functions (host, FP64).
//
// Problem (Section 3.3, Eq. csum2 and Eq. norm_bound): for width W and
// cropping parameter x0, find the even function C supported on [-W/2, W/2]
// and the real correction h minimising
//   E^2 = 1/(2 x0) int_{-x0}^{x0} int_{-1/2}^{1/2} |L(x, nu)|^2 dnu dx,
//   L(x, nu) = 1 - h(x) sum_s C(s - nu) exp(2 pi i (s - nu) x),
// s = -(W-1)/2 .. (W-1)/2.
//
// Method.  Write c_s(nu) = C(s - nu).  For fixed h the best c(nu) solves a
// least-squares problem whose normal matrix is independent of nu, so each
// c_s is an entire function of nu and a Chebyshev series in 2 nu of modest
// degree represents it to rounding level.  For fixed c the best h is
// pointwise, h(x) = int Re a dnu / int |a|^2 dnu with a = sum_s c_s(nu)
// exp(2 pi i (s - nu) x).  Substituting that h leaves a small-residual
// nonlinear least-squares problem in the Chebyshev coefficients, solved by
// Gauss-Newton with Householder QR and a backtracking line search (for large
// x0 followed up from x0 = 1/4).
// Evenness C(u) = C(-u) is built in: c_{-s}(nu) = c_s(-nu).
#include "lmfit.hpp"

#include <algorithm>
#include <cmath>
#include <complex>

namespace ws {
namespace {

constexpr double kPi = 3.14159265358979323846;
using cplx = std::complex<double>;

void gauss_legendre(int n, double a, double b, std::vector<double> *x, std::vector<double> *w) {
    x->assign(n, 0.0);
    w->assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        (*x)[i] = 0.5 * (b - a) * t + 0.5 * (b + a);
        (*w)[i] = (b - a) / ((1.0 - t * t) * dp * dp);
    }
}

void chebyshev_T(double y, int deg, double *T) {
    T[0] = 1.0;
    if (deg >= 1) T[1] = y;
    for (int k = 2; k <= deg; ++k) T[k] = 2.0 * y * T[k - 1] - T[k - 2];
}

// Householder least squares: minimise |A x - b|, A m x n column-major, m >= n.
// A and b are overwritten.  Returns false if a column is numerically zero.
bool householder_lstsq(int m, int n, std::vector<double> &A, std::vector<double> &b,
                       std::vector<double> *x) {
    std::vector<double> diag(n);
    for (int j = 0; j < n; ++j) {
        double *col = &A[(size_t)j * m];
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += col[i] * col[i];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return false;
        double alpha = col[j] > 0 ? -nrm : nrm;
        col[j] -= alpha;                       // v = col - alpha e_j (stored in place)
        double vnorm2 = 0.0;
        for (int i = j; i < m; ++i) vnorm2 += col[i] * col[i];
        for (int k = j + 1; k < n; ++k) {
            double *ck = &A[(size_t)k * m];
            double dot = 0.0;
            for (int i = j; i < m; ++i) dot += col[i] * ck[i];
            double f = 2.0 * dot / vnorm2;
            for (int i = j; i < m; ++i) ck[i] -= f * col[i];
        }
        double dot = 0.0;
        for (int i = j; i < m; ++i) dot += col[i] * b[i];
        double f = 2.0 * dot / vnorm2;
        for (int i = j; i < m; ++i) b[i] -= f * col[i];
        diag[j] = alpha;
    }
    x->assign(n, 0.0);
    for (int j = n - 1; j >= 0; --j) {
        double s = b[j];
        for (int k = j + 1; k < n; ++k) s -= A[(size_t)k * m + j] * (*x)[k];
        (*x)[j] = s / diag[j];
    }
    return true;
}

struct Problem {
    int W, D, nx, nn, npar;
    double x0;
    std::vector<double> xq, wx, nq, wn;
    std::vector<int> tap, kk;                 // parameter p -> (tap i >= centre, degree k)
    std::vector<cplx> dA;                     // npar x nx x nn: d a(x, nu) / d param
};

double tap_offset(int W, int i) { return i - 0.5 * (W - 1); }

void build_problem(int W, double x0, int D, int nx, int nn, Problem *P) {
    P->W = W;
    P->D = D;
    P->nx = nx;
    P->nn = nn;
    P->x0 = x0;
    gauss_legendre(nx, -x0, x0, &P->xq, &P->wx);
    gauss_legendre(nn, -0.5, 0.5, &P->nq, &P->wn);
    P->tap.clear();
    P->kk.clear();
    for (int i = 0; i < W; ++i) {
        double s = tap_offset(W, i);
        if (s < 0) continue;
        for (int k = 0; k <= D; ++k) {
            if (s == 0.0 && (k & 1)) continue;  // c_0 is even in nu
            P->tap.push_back(i);
            P->kk.push_back(k);
        }
    }
    P->npar = (int)P->tap.size();
    P->dA.assign((size_t)P->npar * nx * nn, cplx(0, 0));
    std::vector<double> T(D + 1);
    for (int j = 0; j < nn; ++j) {
        double nu = P->nq[j];
        chebyshev_T(2.0 * nu, D, T.data());
        for (int q = 0; q < nx; ++q) {
            double x = P->xq[q];
            for (int p = 0; p < P->npar; ++p) {
                int i = P->tap[p], k = P->kk[p];
                int mirror = W - 1 - i;
                double s = tap_offset(W, i);
                cplx v = T[k] * std::polar(1.0, 2 * kPi * (s - nu) * x);
                if (mirror != i) {
                    double sm = tap_offset(W, mirror);
                    double sign = (k & 1) ? -1.0 : 1.0;  // T_k(-y) = (-1)^k T_k(y)
                    v += sign * T[k] * std::polar(1.0, 2 * kPi * (sm - nu) * x);
                }
                P->dA[((size_t)p * nx + q) * nn + j] = v;
            }
        }
    }
}

struct State {
    std::vector<cplx> a;                 // nx x nn
    std::vector<double> R, Q, h;         // nx
    double obj = 0.0;
};

void evaluate(const Problem &P, const std::vector<double> &beta, State *S) {
    const int nx = P.nx, nn = P.nn;
    S->a.assign((size_t)nx * nn, cplx(0, 0));
    for (int p = 0; p < P.npar; ++p) {
        const cplx *src = &P.dA[(size_t)p * nx * nn];
        for (size_t e = 0; e < (size_t)nx * nn; ++e) S->a[e] += beta[p] * src[e];
    }
    S->R.assign(nx, 0.0);
    S->Q.assign(nx, 0.0);
    S->h.assign(nx, 0.0);
    double obj = 0.0;
    for (int q = 0; q < nx; ++q) {
        double R = 0.0, Q = 0.0;
        for (int j = 0; j < nn; ++j) {
            cplx a = S->a[(size_t)q * nn + j];
            R += P.wn[j] * a.real();
            Q += P.wn[j] * std::norm(a);
        }
        double h = R / Q;
        S->R[q] = R;
        S->Q[q] = Q;
        S->h[q] = h;
        for (int j = 0; j < nn; ++j) {
            cplx rho = 1.0 - h * S->a[(size_t)q * nn + j];
            obj += P.wx[q] * P.wn[j] * std::norm(rho);
        }
    }
    S->obj = obj / (2.0 * P.x0);
}

}  // namespace

void tap_weights(const LeastMisfitFit &f, double nu, double *c) {
    std::vector<double> T(f.degree + 1);
    chebyshev_T(2.0 * nu, f.degree, T.data());
    for (int i = 0; i < f.W; ++i) {
        double s = 0.0;
        for (int k = 0; k <= f.degree; ++k) s += f.cheb[(size_t)i * (f.degree + 1) + k] * T[k];
        c[i] = s;
    }
}

double h_direct(const LeastMisfitFit &f, double x) {
    static thread_local std::vector<double> nq, wn;
    if ((int)nq.size() != 80) gauss_legendre(80, -0.5, 0.5, &nq, &wn);
    std::vector<double> c(f.W);
    double R = 0.0, Q = 0.0;
    for (size_t j = 0; j < nq.size(); ++j) {
        tap_weights(f, nq[j], c.data());
        cplx a(0, 0);
        for (int i = 0; i < f.W; ++i) a += c[i] * std::polar(1.0, 2 * kPi * (tap_offset(f.W, i) - nq[j]) * x);
        R += wn[j] * a.real();
        Q += wn[j] * std::norm(a);
    }
    return R / Q;
}

double h_series(const LeastMisfitFit &f, double x) {
    // Clenshaw recurrence for sum_k h_cheb[k] T_k(x / x0)
    double y = x / f.x0, b1 = 0.0, b2 = 0.0;
    for (int k = f.h_terms - 1; k >= 1; --k) {
        double b0 = 2.0 * y * b1 - b2 + f.h_cheb[k];
        b2 = b1;
        b1 = b0;
    }
    return y * b1 - b2 + f.h_cheb[0];
}

namespace {

// Damped Gauss-Newton on the coefficients of one problem, from beta (or, if
// beta is empty, from the best c for h = 1).  The misfit is unchanged by
// beta -> alpha beta (h scales as 1 / alpha), so the Jacobian has the null
// direction beta; one extra row asks the step to be orthogonal to beta,
// which removes it without damping any other direction.  Each step is
// halved until E^2 falls.
bool gauss_newton(const Problem &P, std::vector<double> *beta_io, std::string *err) {
    const int nx = P.nx, nn = P.nn, npar = P.npar;
    const int m = 2 * nx * nn;
    std::vector<double> sq((size_t)nx * nn);
    for (int q = 0; q < nx; ++q)
        for (int j = 0; j < nn; ++j) sq[(size_t)q * nn + j] = std::sqrt(P.wx[q] * P.wn[j]);
    std::vector<double> &beta = *beta_io;
    if (beta.empty()) {
        // Start: best c for h = 1, i.e. minimise sum w |1 - a|^2 (linear in beta).
        std::vector<double> A((size_t)m * npar), b(m, 0.0);
        for (int p = 0; p < npar; ++p)
            for (size_t e = 0; e < (size_t)nx * nn; ++e) {
                cplx v = sq[e] * P.dA[(size_t)p * nx * nn + e];
                A[(size_t)p * m + e] = v.real();
                A[(size_t)p * m + nx * nn + e] = v.imag();
            }
        for (size_t e = 0; e < (size_t)nx * nn; ++e) b[e] = sq[e];
        if (!householder_lstsq(m, npar, A, b, &beta)) {
            *err = "least-misfit fit: singular start";
            return false;
        }
    }
    State S, C;
    evaluate(P, beta, &S);
    const int rows = m + 1;
    std::vector<double> J((size_t)rows * npar), r(rows), step;
    std::vector<double> dR((size_t)npar * nx), dQ((size_t)npar * nx);
    for (int iter = 0; iter < 80; ++iter) {
        // Jacobian of rho = 1 - h a with h = R/Q.
        for (int p = 0; p < npar; ++p)
            for (int q = 0; q < nx; ++q) {
                double sr = 0.0, sqq = 0.0;
                for (int j = 0; j < nn; ++j) {
                    cplx d = P.dA[((size_t)p * nx + q) * nn + j];
                    cplx a = S.a[(size_t)q * nn + j];
                    sr += P.wn[j] * d.real();
                    sqq += 2.0 * P.wn[j] * (std::conj(a) * d).real();
                }
                dR[(size_t)p * nx + q] = sr;
                dQ[(size_t)p * nx + q] = sqq;
            }
        double colmax = 0.0, bnorm = 0.0;
        for (int p = 0; p < npar; ++p) {
            double cn = 0.0;
            for (int q = 0; q < nx; ++q) {
                double dh = dR[(size_t)p * nx + q] / S.Q[q] -
                            S.R[q] / (S.Q[q] * S.Q[q]) * dQ[(size_t)p * nx + q];
                for (int j = 0; j < nn; ++j) {
                    size_t e = (size_t)q * nn + j;
                    cplx v = -(dh * S.a[e] + S.h[q] * P.dA[(size_t)p * nx * nn + e]) * sq[e];
                    J[(size_t)p * rows + e] = v.real();
                    J[(size_t)p * rows + nx * nn + e] = v.imag();
                    cn += std::norm(v);
                }
            }
            colmax = std::max(colmax, cn);
            bnorm += beta[p] * beta[p];
        }
        // the gauge row: sqrt(colmax) beta / |beta| . step = 0
        bnorm = std::sqrt(bnorm);
        for (int p = 0; p < npar; ++p) J[(size_t)p * rows + m] = std::sqrt(colmax) * beta[p] / bnorm;
        for (int q = 0; q < nx; ++q)
            for (int j = 0; j < nn; ++j) {
                size_t e = (size_t)q * nn + j;
                cplx rho = (1.0 - S.h[q] * S.a[e]) * sq[e];
                r[e] = -rho.real();
                r[nx * nn + e] = -rho.imag();
            }
        r[m] = 0.0;
        if (!householder_lstsq(rows, npar, J, r, &step)) break;
        double lam = 1.0;
        bool improved = false;
        std::vector<double> trial(npar);
        while (lam > 1e-8) {
            for (int p = 0; p < npar; ++p) trial[p] = beta[p] + lam * step[p];
            evaluate(P, trial, &C);
            if (C.obj < S.obj) {
                improved = true;
                break;
            }
            lam *= 0.5;
        }
        if (!improved) break;
        double rel = (S.obj - C.obj) / S.obj;
        beta = trial;
        std::swap(S, C);
        if (rel < 1e-9) break;
    }
    return true;
}

}  // namespace

bool fit_least_misfit(int W, double x0, LeastMisfitFit *out, std::string *err) {
    if (W < 1 || W > 16 || !(x0 > 0.0) || x0 > 0.5) {
        *err = "least-misfit fit needs 1 <= W <= 16 and 0 < x0 <= 0.5";
        return false;
    }
    const int D = 18, nx = 48, nn = 48;
    // Above x0 = 0.3 the minimiser is followed up from x0 = 1/4 in steps of
    // 0.05, each fit starting from the last one's coefficients: started cold
    // at large x0, Gauss-Newton can settle in a much poorer local minimum.
    std::vector<double> path{x0};
    if (x0 > 0.3) {
        path.assign(1, 0.25);
        while (path.back() + 0.05 < x0 - 1e-12) path.push_back(path.back() + 0.05);
        path.push_back(x0);
    }
    Problem P;
    std::vector<double> beta;
    for (double xs : path) {
        build_problem(W, xs, D, nx, nn, &P);
        if (!gauss_newton(P, &beta, err)) return false;
    }
    const int npar = P.npar;

    LeastMisfitFit f;
    f.W = W;
    f.x0 = x0;
    f.degree = D;
    f.cheb.assign((size_t)W * (D + 1), 0.0);
    for (int p = 0; p < npar; ++p) {
        int i = P.tap[p], k = P.kk[p], mirror = W - 1 - i;
        f.cheb[(size_t)i * (D + 1) + k] += beta[p];
        if (mirror != i) f.cheb[(size_t)mirror * (D + 1) + k] += ((k & 1) ? -1.0 : 1.0) * beta[p];
    }
    // Gauge: scale so that h(0) = 1 (h scales as 1 / C).
    double h0 = h_direct(f, 0.0);
    for (double &v : f.cheb) v *= h0;

    // Chebyshev series of h on [-x0, x0] from Chebyshev-node samples.
    const int nh = 48;
    std::vector<double> hv(nh);
    for (int j = 0; j < nh; ++j) hv[j] = h_direct(f, x0 * std::cos(kPi * (j + 0.5) / nh));
    f.h_terms = nh;
    f.h_cheb.assign(nh, 0.0);
    for (int k = 0; k < nh; ++k) {
        double s = 0.0;
        for (int j = 0; j < nh; ++j) s += hv[j] * std::cos(kPi * k * (j + 0.5) / nh);
        f.h_cheb[k] = (k == 0 ? 1.0 : 2.0) * s / nh;
    }
    double herr = 0.0;
    for (int j = 0; j <= 64; ++j) {
        double x = x0 * (-1.0 + 2.0 * j / 64.0);
        double hd = h_direct(f, x);
        herr = std::max(herr, std::fabs(h_series(f, x) - hd) / std::fabs(hd));
    }
    f.h_interp_err = herr;

    // E on a finer quadrature than the fit used.
    std::vector<double> xf, wxf, nf, wnf;
    gauss_legendre(96, -x0, x0, &xf, &wxf);
    gauss_legendre(96, -0.5, 0.5, &nf, &wnf);
    std::vector<std::vector<double>> cw(nf.size(), std::vector<double>(W));
    for (size_t j = 0; j < nf.size(); ++j) tap_weights(f, nf[j], cw[j].data());
    double e2 = 0.0;
    for (size_t q = 0; q < xf.size(); ++q) {
        double h = h_series(f, xf[q]);
        for (size_t j = 0; j < nf.size(); ++j) {
            cplx a(0, 0);
            for (int i = 0; i < W; ++i)
                a += cw[j][i] * std::polar(1.0, 2 * kPi * (tap_offset(W, i) - nf[j]) * xf[q]);
            e2 += wxf[q] * wnf[j] * std::norm(1.0 - h * a);
        }
    }
    f.E = std::sqrt(e2 / (2.0 * x0));
    *out = f;
    return true;
}

void monomial_weights(const LeastMisfitFit &f, double tol, int max_deg, int *deg,
                      std::vector<double> *out) {
    const int D = f.degree;
    // T_k(y) in powers of y, then y = 2 nu.
    std::vector<std::vector<double>> Tm(D + 1, std::vector<double>(D + 1, 0.0));
    Tm[0][0] = 1.0;
    if (D >= 1) Tm[1][1] = 1.0;
    for (int k = 2; k <= D; ++k)
        for (int p = 0; p <= k; ++p)
            Tm[k][p] = (p > 0 ? 2.0 * Tm[k - 1][p - 1] : 0.0) - Tm[k - 2][p];
    std::vector<double> mono((size_t)f.W * (D + 1), 0.0);
    for (int i = 0; i < f.W; ++i)
        for (int k = 0; k <= D; ++k)
            for (int p = 0; p <= k; ++p)
                mono[(size_t)i * (D + 1) + p] += f.cheb[(size_t)i * (D + 1) + k] * Tm[k][p] * std::ldexp(1.0, p);
    int d = std::min(D, max_deg);
    while (d > 0) {
        double tail = 0.0;
        for (int i = 0; i < f.W; ++i)
            tail = std::max(tail, std::fabs(mono[(size_t)i * (D + 1) + d]) * std::ldexp(1.0, -d));
        if (tail > tol) break;
        --d;
    }
    *deg = d;
    out->assign((size_t)f.W * (d + 1), 0.0);
    for (int i = 0; i < f.W; ++i)
        for (int p = 0; p <= d; ++p) (*out)[(size_t)i * (d + 1) + p] = mono[(size_t)i * (D + 1) + p];
}

}  // namespace ws
