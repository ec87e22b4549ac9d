// Plan-time least-misfit gridding functions (host, FP64).
//
// The pair (C, h) minimises the error bound E of Eq. norm_bound (Section 3.3)
// for a kernel width W and cropping parameter x0; its definition is the
// "Making a map" box of Section 3.3.  See lmfit.cpp for the method.
#pragma once

#include <string>
#include <vector>

namespace ws {

struct LeastMisfitFit {
    int W = 0;
    double x0 = 0.0;
    int degree = 0;                 // Chebyshev degree of each tap function
    std::vector<double> cheb;       // W x (degree+1): c_i(nu) = sum_k cheb[i][k] T_k(2 nu)
    int h_terms = 0;
    std::vector<double> h_cheb;     // Chebyshev series of h on [-x0, x0] (argument x/x0)
    double E = 0.0;                 // error bound of Eq. norm_bound
    double h_interp_err = 0.0;      // max relative error of the h series at check points
};

// Fit the least-misfit pair.  Returns false and sets *err on failure.
bool fit_least_misfit(int W, double x0, LeastMisfitFit *out, std::string *err);

// c_i(nu) for all W taps at one nu in [-1/2, 1/2].
void tap_weights(const LeastMisfitFit &f, double nu, double *c);

// h(x) straight from the fit (ratio of nu-integrals); slow, used for checks.
double h_direct(const LeastMisfitFit &f, double x);

// h(x) from its Chebyshev series, |x| <= x0.
double h_series(const LeastMisfitFit &f, double x);

// Monomial coefficients of c_i(nu) in nu: out[i*(deg+1) + m] multiplies nu^m.
// deg is the smallest degree whose dropped tail stays below tol on |nu|<=1/2.
void monomial_weights(const LeastMisfitFit &f, double tol, int max_deg, int *deg,
                      std::vector<double> *out);

}  // namespace ws
