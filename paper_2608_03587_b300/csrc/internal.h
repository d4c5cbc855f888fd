// Internal declarations shared by the host assembly and the CUDA side of
// libdecbpm.  Not part of the C ABI.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "decbpm.h"

namespace decbpm {

// Thread-local error message; fail() records it and returns `code`.
int fail(int code, const char *fmt, ...);
void clear_error();

// FP64 host assembly of one mesh.  Everything is in the caller's vertex order
// except perm/iperm, which define the internal (reverse Cuthill-McKee) order.
struct Assembly {
    int dim = 2;
    int64_t n0 = 0, nc = 0, n_edges = 0;
    std::vector<double> m;        // *0 (barycentric dual cell measure)
    std::vector<double> v;        // *0^{-1} *0(V) 1: lumped potential
    std::vector<double> chib;     // *0^{-1} *0(chi) 1: lumped Kerr coefficient
    std::vector<double> sigma;    // absorber rate
    std::vector<double> p;        // diffraction coefficients p_1..p_n
    // off-diagonal stiffness pattern, CSR, neighbours ascending:
    //   K_pq = -w[pq] for q != p, K_pp = wsum[p] = sum_q w_pq
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> w;        // edge weights (cotangent form of d0^T *1 d0)
    std::vector<double> wsum;
    // element-averaged Kerr operator C = *0^{-1} Q^T D Q (Eq. 14), same pattern
    std::vector<double> c_off;
    std::vector<double> c_diag;
    double rho = 0.0;             // upper end of the Chebyshev interval of A = *0^{-1} K (see rho_kind)
    double rho_gershgorin = 0.0;  // max_p (sum_q w_pq + sum_q |w_pq|) / m_p
    double rho_element = 0.0;     // max_t lambda_max(K_t, M_t)
    double rho_lanczos = 0.0;     // largest Ritz value of the Lanczos steps (0 if not run)
    double rho_rigorous = 0.0;    // (1 + 1e-6) min(Gershgorin, element bound)
    int32_t rho_kind = DECBPM_RHO_RIGOROUS;   // which bound rho is (DECBPM_RHO_*)
    double area = 0.0;
    int32_t max_degree = 0;
    std::vector<int32_t> perm;    // perm[new] = old
    std::vector<int32_t> iperm;   // iperm[old] = new
    int64_t bandwidth = 0;
};

int assemble(const decbpm_mesh_desc *desc, Assembly &out);

// SELL-32 packing of the off-diagonal pattern in internal order.  Slice s
// holds rows 32s..32s+31; entry (row, j) sits at slice_ptr[s] + 32 j + lane.
// Padding entries point at their own row with zero weight.
constexpr int kSlice = 32;
struct Sell {
    int64_t n_rows = 0, n_slices = 0;
    std::vector<int32_t> slice_ptr;   // [n_slices + 1]
    std::vector<int32_t> slice_w;     // [n_slices]
    std::vector<int32_t> col;         // internal column index
    std::vector<double> w;            // w_pq (0 for padding)
    std::vector<double> c;            // element-Kerr c_pq (0 for padding)
    std::vector<int32_t> degree;      // [n_rows] true off-diagonal count
};
void build_sell(const Assembly &a, Sell &s);

// Bessel J_0..J_kmax(a) (a >= 0) by Miller's backward recurrence.
void bessel_sequence(double a, int kmax, double *J);

// Scaled modified Bessel functions s_k = e^{-a} I_k(a), k = 0..M, a >= 0, by
// Miller's backward recurrence normalised with I_0 + 2 sum_k I_k = e^a; M is
// the first index from which every s_k < tol s_0.  They give the Chebyshev
// series e^{-a x} = e^{a} [s_0 + 2 sum_k (-1)^k s_k T_k(x)] on [-1, 1].
void bessel_i_scaled(double a, double tol, std::vector<double> &s);

// Chebyshev expansion of f(lambda) = exp(i h g(lambda)), g = sum_n p_n (-lambda)^n,
// on [0, rho] in x = (lambda - c) / r, c = r = rho / 2:
//     f = exp(i theta0) sum_k a_k T_k(x),   theta0 = h g(c).
// The constant phase theta0 is kept out of a_k: rounding it into FP32
// coefficients would add the same phase error at every step.
struct Cheb {
    int M = 0;                                  // degree (>= 2)
    double theta0 = 0.0;
    std::complex<double> f0;                    // exact f(lambda = 0) e^{-i theta0}
    std::vector<std::complex<double>> a;        // a_0 .. a_M
};
int cheb_coefficients(const std::vector<double> &p, double rho, double h, double tol, Cheb &out);

}  // namespace decbpm
