// Host-side FP64 assembly of the DEC operators, vertex renumbering, SELL
// packing and Chebyshev coefficients.
//
// Operators (Sec. "DEC computational framework", "Discrete Hodge star"):
//   * edges [v_a, v_b] with a < b; d0 has +1 at the head v_b, -1 at the tail;
//   * *0: m_p = (1/(d+1)) sum_{t ni p} |t|  (1/3 for triangles, 1/2 for segments);
//   * *0(V), *0(chi): the same sums weighted by the per-cell value;
//   * d0^T *1 d0 with the Galerkin *1 of Eq. 9 (Whitney 1-forms, xi = 1) is the
//     P1 stiffness matrix, whose off-diagonal entries are -w_e with the
//     cotangent weight w_e = (1/2) sum over the triangles at e of the cotangent
//     of the angle opposite e (1/|e| in 1D).  Only w_e is stored: K_pq = -w_pq,
//     K_pp = sum_q w_pq.
//   * element-averaged Kerr (Eqs. 13-14): *0^{-1} Q^T D Q with Q = (1/6)|d1||d0|
//     has entries c_pq = (1/(9 m_p)) sum_{t ni p,q} chi_t |t| and
//     c_pp = (1/(9 m_p)) sum_{t ni p} chi_t |t|  ((d+1)^2 in place of 9 in 1D).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace decbpm {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

const char *last_error_cstr() { return g_err.c_str(); }

static bool finite_all(const double *x, int64_t n) {
    if (!x) return true;
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

// Reverse Cuthill-McKee on the CSR pattern.  Each connected component starts
// from a pseudo-peripheral vertex (repeated BFS, George-Liu), neighbours are
// enqueued by increasing degree, and the final order is reversed.
static void rcm(const std::vector<int64_t> &rowptr, const std::vector<int32_t> &col, int64_t n,
                std::vector<int32_t> &perm) {
    std::vector<int32_t> deg(n);
    for (int64_t i = 0; i < n; ++i) deg[i] = int32_t(rowptr[i + 1] - rowptr[i]);
    std::vector<int32_t> level(n, -1);
    std::vector<char> placed(n, 0);
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<int32_t> queue(n), nb;

    auto bfs_levels = [&](int32_t root, std::vector<int32_t> &touched) -> int32_t {
        // returns the last vertex of the deepest level with minimal degree
        int64_t head = 0, tail = 0;
        queue[tail++] = root;
        level[root] = 0;
        touched.push_back(root);
        int32_t maxlev = 0;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
                int32_t w = col[k];
                if (level[w] < 0 && !placed[w]) {
                    level[w] = level[u] + 1;
                    maxlev = std::max(maxlev, level[w]);
                    queue[tail++] = w;
                    touched.push_back(w);
                }
            }
        }
        int32_t best = root;
        for (int32_t t : touched)
            if (level[t] == maxlev && (best == root || deg[t] < deg[best])) best = t;
        return best;
    };

    for (int64_t s = 0; s < n; ++s) {
        if (placed[s]) continue;
        // pseudo-peripheral start of this component
        int32_t root = int32_t(s);
        int32_t ecc = -1;
        for (int it = 0; it < 6; ++it) {
            std::vector<int32_t> touched;
            int32_t far = bfs_levels(root, touched);
            int32_t e = level[far];
            for (int32_t t : touched) level[t] = -1;
            if (e <= ecc) break;
            ecc = e;
            root = far;
        }
        // Cuthill-McKee BFS
        int64_t head = 0, tail = 0;
        queue[tail++] = root;
        placed[root] = 1;
        while (head < tail) {
            int32_t u = queue[head++];
            order.push_back(u);
            nb.clear();
            for (int64_t k = rowptr[u]; k < rowptr[u + 1]; ++k)
                if (!placed[col[k]]) nb.push_back(col[k]);
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            for (int32_t w : nb) {
                placed[w] = 1;
                queue[tail++] = w;
            }
        }
    }
    std::reverse(order.begin(), order.end());
    perm.assign(order.begin(), order.end());
}

// Position of (x, y) on the Hilbert curve filling a 2^order x 2^order grid
// (the iterative rotate-and-reflect construction).
static uint64_t hilbert_index(uint32_t x, uint32_t y, int order) {
    uint64_t d = 0;
    for (uint32_t s = 1u << (order - 1); s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u;
        const uint32_t ry = (y & s) ? 1u : 0u;
        d += uint64_t(s) * uint64_t(s) * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) { x = s - 1 - (x & (s - 1)) + (x & ~(s - 1)); y = s - 1 - (y & (s - 1)) + (y & ~(s - 1)); }
            std::swap(x, y);
        }
    }
    return d;
}

// Vertices sorted along a Hilbert curve of their (quantized) positions; in
// 1D, by coordinate.
static void hilbert_order(const double *X, int dim, int64_t n, std::vector<int32_t> &perm) {
    std::vector<std::pair<uint64_t, int32_t>> key(n);
    double lo[2] = {X[0], dim == 2 ? X[1] : 0.0}, hi[2] = {X[0], dim == 2 ? X[1] : 0.0};
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < dim; ++a) { lo[a] = std::min(lo[a], X[i * dim + a]); hi[a] = std::max(hi[a], X[i * dim + a]); }
    const int order = 20;
    const double span = std::max(hi[0] - lo[0], dim == 2 ? hi[1] - lo[1] : 0.0);
    const double scale = span > 0 ? double((1u << order) - 1) / span : 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t qx = uint32_t((X[i * dim] - lo[0]) * scale);
        if (dim == 1) { key[i] = {qx, int32_t(i)}; continue; }
        const uint32_t qy = uint32_t((X[i * dim + 1] - lo[1]) * scale);
        key[i] = {hilbert_index(qx, qy, order), int32_t(i)};
    }
    std::sort(key.begin(), key.end());
    perm.resize(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = key[i].second;
}

// Largest eigenvalue of the symmetric tridiagonal matrix (diag a, off b) by
// bisection on the Sturm count.
static double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &b) {
    const int k = int(a.size());
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto count_above = [&](double x) {      // eigenvalues > x
        int neg = 0;
        double q = a[0] - x;
        if (q < 0) ++neg;
        for (int i = 1; i < k; ++i) {
            const double qq = q == 0.0 ? 1e-300 : q;
            q = a[i] - x - b[i - 1] * b[i - 1] / qq;
            if (q < 0) ++neg;
        }
        return k - neg;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_above(mid) >= 1) lo = mid;
        else hi = mid;
    }
    return hi;
}

// Lanczos estimate of lambda_max(*0^{-1} K) = lambda_max(S), S = *0^{-1/2} K *0^{-1/2}
// symmetric, from a fixed pseudo-random start (no reorthogonalization: the
// largest Ritz value still converges to lambda_max from below).
static double lanczos_lambda_max(const Assembly &A, int steps) {
    const int64_t n = A.n0;
    std::vector<double> isq(n), v(n), vprev(n, 0.0), w(n), tmp(n);
    for (int64_t i = 0; i < n; ++i) isq[i] = 1.0 / std::sqrt(A.m[i]);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;                  // xorshift64
        v[i] = double(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        nrm += v[i] * v[i];
    }
    nrm = std::sqrt(nrm);
    for (auto &x : v) x /= nrm;
    std::vector<double> alpha, beta;
    double bprev = 0.0;
    const int k = int(std::min<int64_t>(steps, n));
    for (int j = 0; j < k; ++j) {
        for (int64_t i = 0; i < n; ++i) tmp[i] = isq[i] * v[i];
        for (int64_t p = 0; p < n; ++p) {                               // w = S v
            double acc = A.wsum[p] * tmp[p];
            for (int64_t e = A.rowptr[p]; e < A.rowptr[p + 1]; ++e) acc -= A.w[e] * tmp[A.col[e]];
            w[p] = isq[p] * acc;
        }
        double a = 0.0;
        for (int64_t i = 0; i < n; ++i) a += w[i] * v[i];
        double b = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            w[i] -= a * v[i] + bprev * vprev[i];
            b += w[i] * w[i];
        }
        b = std::sqrt(b);
        alpha.push_back(a);
        if (j + 1 == k || b < 1e-300) break;
        beta.push_back(b);
        for (int64_t i = 0; i < n; ++i) {
            vprev[i] = v[i];
            v[i] = w[i] / b;
        }
        bprev = b;
    }
    beta.resize(alpha.size() > 0 ? alpha.size() - 1 : 0);
    return tridiag_max_eig(alpha, beta);
}

// Deterministic check that no eigenvalue of S = *0^{-1/2} K *0^{-1/2} (the
// spectrum of A) lies above a candidate rho.  With rho_t = rho / 1.002 and
// X = 2 S / rho_t - 1, every eigenvalue in [0, rho_t] has |T_k(x)| <= 1, so
// ||T_k(X) z|| <= ||z|| for every vector z and every degree k.  An eigenvalue
// lambda > rho_t (x > 1) instead contributes T_k(x) |c| with
// T_k(x) = cosh(k acosh x), c its component in z.  The probe z is a seeded
// pseudo-random vector (a generator and seed of its own, not the Lanczos
// start) plus unit spikes at the 8 vertices whose Gershgorin rows are largest
// (where the top eigenvectors of graded meshes concentrate).  Passing at degree
// 128 therefore shows that every eigenvector whose component in z is at least
// 1e-3 of ||z|| has lambda < rho (T_128 = 1000 at x = 1.00176, i.e. at
// rho_t * 1.00088 < rho).  It is no proof for an eigenvector orthogonal to z to
// that accuracy; no probability is claimed for it.
static bool verify_upper_bound(const Assembly &A, double rho, int degree) {
    const int64_t n = A.n0;
    const double rho_t = rho / 1.002;
    std::vector<double> isq(n), z(n), t0(n), t1(n), t2(n), tmp(n);
    for (int64_t i = 0; i < n; ++i) isq[i] = 1.0 / std::sqrt(A.m[i]);
    uint64_t st = 0xD1B54A32D192ED03ull;            // splitmix64, a different stream from the Lanczos start
    double nr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t x = st;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        z[i] = double(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        nr += z[i] * z[i];
    }
    for (auto &x : z) x /= std::sqrt(nr);
    // spikes at the largest Gershgorin rows of A
    std::vector<std::pair<double, int64_t>> g(n);
    for (int64_t p = 0; p < n; ++p) {
        double wabs = 0.0;
        for (int64_t e = A.rowptr[p]; e < A.rowptr[p + 1]; ++e) wabs += std::fabs(A.w[e]);
        g[p] = {(A.wsum[p] + wabs) / A.m[p], p};
    }
    const int64_t n_spikes = std::min<int64_t>(8, n);
    std::partial_sort(g.begin(), g.begin() + n_spikes, g.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    for (int64_t j = 0; j < n_spikes; ++j) z[g[j].second] += 1.0;
    double z2 = 0.0;
    for (double x : z) z2 += x * x;
    auto apply_X = [&](const std::vector<double> &u, std::vector<double> &out) {
        for (int64_t i = 0; i < n; ++i) tmp[i] = isq[i] * u[i];
        for (int64_t p = 0; p < n; ++p) {
            double acc = A.wsum[p] * tmp[p];
            for (int64_t e = A.rowptr[p]; e < A.rowptr[p + 1]; ++e) acc -= A.w[e] * tmp[A.col[e]];
            out[p] = (2.0 / rho_t) * isq[p] * acc - u[p];
        }
    };
    const double limit = (1.0 + 1e-8) * (1.0 + 1e-8) * z2;
    t0 = z;
    apply_X(t0, t1);
    for (int k = 1; k < degree; ++k) {
        double s2 = 0.0;
        for (double x : t1) s2 += x * x;
        if (!(s2 <= limit)) return false;            // also catches NaN
        apply_X(t1, t2);
        for (int64_t i = 0; i < n; ++i) t2[i] = 2.0 * t2[i] - t0[i];
        std::swap(t0, t1);
        std::swap(t1, t2);
    }
    double s2 = 0.0;
    for (double x : t1) s2 += x * x;
    return s2 <= limit;
}

int assemble(const decbpm_mesh_desc *d, Assembly &A) {
    if (!d) return fail(DECBPM_ERR_INVALID_ARG, "mesh description is NULL");
    if (d->dim != 1 && d->dim != 2) return fail(DECBPM_ERR_INVALID_ARG, "dim must be 1 or 2 (got %d)", d->dim);
    if (d->n_vertices < 2 || d->n_cells < 1)
        return fail(DECBPM_ERR_INVALID_ARG, "need >= 2 vertices and >= 1 cell");
    if (d->n_vertices > (int64_t(1) << 30))
        return fail(DECBPM_ERR_INVALID_ARG, "n_vertices %lld exceeds 2^30", (long long)d->n_vertices);
    if (!d->coords || !d->cells) return fail(DECBPM_ERR_INVALID_ARG, "coords and cells are required");
    if (d->n_p < 0 || (d->n_p > 0 && !d->p_n)) return fail(DECBPM_ERR_INVALID_ARG, "bad p_n / n_p");
    const int dim = d->dim, kv = dim + 1;
    const int64_t n0 = d->n_vertices, nc = d->n_cells;
    if (!finite_all(d->coords, n0 * dim)) return fail(DECBPM_ERR_NONFINITE, "non-finite coordinate");
    if (!finite_all(d->V_cell, nc) || !finite_all(d->chi_cell, nc) || !finite_all(d->sigma_vertex, n0) ||
        !finite_all(d->p_n, d->n_p))
        return fail(DECBPM_ERR_NONFINITE, "non-finite material, absorber or p_n value");
    for (int64_t i = 0; d->sigma_vertex && i < n0; ++i)
        if (d->sigma_vertex[i] < 0) return fail(DECBPM_ERR_INVALID_ARG, "sigma_vertex[%lld] < 0", (long long)i);
    for (int64_t i = 0; i < nc * kv; ++i)
        if (d->cells[i] < 0 || d->cells[i] >= n0)
            return fail(DECBPM_ERR_BAD_MESH, "cell vertex index out of range at cells[%lld]", (long long)i);

    A = Assembly();
    A.dim = dim;
    A.n0 = n0;
    A.nc = nc;
    if (d->n_p > 0) A.p.assign(d->p_n, d->p_n + d->n_p);
    else A.p = {1.0};
    A.m.assign(n0, 0.0);
    std::vector<double> mV(n0, 0.0), mchi(n0, 0.0), cdiag(n0, 0.0);
    A.sigma.assign(n0, 0.0);
    if (d->sigma_vertex) std::copy(d->sigma_vertex, d->sigma_vertex + n0, A.sigma.begin());

    // one record per (cell, edge): key (a < b), cotangent contribution, chi|t|
    struct Rec { int64_t a, b; double w, c; };
    std::vector<Rec> recs;
    recs.reserve(size_t(nc) * (dim == 2 ? 3 : 1));
    const double *X = d->coords;
    double area = 0.0;
    // element eigenvalue bound: with K = sum_t K_t and *0 = sum_t M_t (M_t the
    // lumped element mass |t|/(d+1) on each vertex of t),
    // x^T K x = sum_t x_t^T K_t x_t <= max_t lambda_max(K_t, M_t) x^T *0 x.
    double rho_elem = 0.0;
    for (int64_t t = 0; t < nc; ++t) {
        const int32_t *c = d->cells + t * kv;
        const double Vt = d->V_cell ? d->V_cell[t] : 0.0;
        const double chit = d->chi_cell ? d->chi_cell[t] : 1.0;
        double meas;
        if (dim == 1) {
            meas = std::fabs(X[c[1]] - X[c[0]]);
            if (!(meas > 0)) return fail(DECBPM_ERR_BAD_MESH, "degenerate segment %lld", (long long)t);
            recs.push_back({std::min<int64_t>(c[0], c[1]), std::max<int64_t>(c[0], c[1]), 1.0 / meas, chit * meas});
            rho_elem = std::max(rho_elem, 4.0 / (meas * meas));      // K_e = [1 -1; -1 1]/L, M_e = L/2
        } else {
            const double *p0 = X + 2 * c[0], *p1 = X + 2 * c[1], *p2 = X + 2 * c[2];
            const double cross = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]);
            if (!(cross > 0))
                return fail(DECBPM_ERR_BAD_MESH, "triangle %lld is %s (cells must be counter-clockwise)",
                            (long long)t, cross < 0 ? "clockwise" : "degenerate");
            meas = 0.5 * cross;
            double wsum_t = 0.0, wprod_t = 0.0, wopp[3];
            for (int i = 0; i < 3; ++i) {
                const int32_t vi = c[i], vj = c[(i + 1) % 3], vk = c[(i + 2) % 3];
                const double *pi = X + 2 * vi, *pj = X + 2 * vj, *pk = X + 2 * vk;
                const double ux = pj[0] - pi[0], uy = pj[1] - pi[1];
                const double wx = pk[0] - pi[0], wy = pk[1] - pi[1];
                const double cot = (ux * wx + uy * wy) / cross;   // |u x w| = cross for CCW
                recs.push_back({std::min<int64_t>(vj, vk), std::max<int64_t>(vj, vk), 0.5 * cot, chit * meas});
                wopp[i] = 0.5 * cot;
                wsum_t += 0.5 * cot;
            }
            // K_t has zero row sums and off-diagonals -w: its nonzero eigenvalues are
            // s +- sqrt(s^2 - 3 (w0 w1 + w1 w2 + w2 w0)), s = w0 + w1 + w2; M_t = |t|/3 I
            wprod_t = wopp[0] * wopp[1] + wopp[1] * wopp[2] + wopp[2] * wopp[0];
            const double disc = std::max(0.0, wsum_t * wsum_t - 3.0 * wprod_t);
            rho_elem = std::max(rho_elem, (wsum_t + std::sqrt(disc)) * 3.0 / meas);
        }
        area += meas;
        for (int i = 0; i < kv; ++i) {
            A.m[c[i]] += meas / kv;
            mV[c[i]] += Vt * meas / kv;
            mchi[c[i]] += chit * meas / kv;
            cdiag[c[i]] += chit * meas;
        }
    }
    A.area = area;
    for (int64_t p = 0; p < n0; ++p)
        if (!(A.m[p] > 0)) return fail(DECBPM_ERR_BAD_MESH, "vertex %lld belongs to no cell", (long long)p);

    std::sort(recs.begin(), recs.end(), [](const Rec &x, const Rec &y) {
        return x.a != y.a ? x.a < y.a : x.b < y.b;
    });
    struct Edge { int64_t a, b; double w, c; };
    std::vector<Edge> E;
    E.reserve(recs.size() / 2 + 1);
    for (size_t i = 0; i < recs.size();) {
        size_t j = i;
        double w = 0, cc = 0;
        while (j < recs.size() && recs[j].a == recs[i].a && recs[j].b == recs[i].b) {
            w += recs[j].w;
            cc += recs[j].c;
            ++j;
        }
        if (j - i > size_t(dim == 2 ? 2 : 1))
            return fail(DECBPM_ERR_BAD_MESH, "edge (%lld, %lld) is shared by %zu cells (non-manifold)",
                        (long long)recs[i].a, (long long)recs[i].b, j - i);
        E.push_back({recs[i].a, recs[i].b, w, cc});
        i = j;
    }
    A.n_edges = int64_t(E.size());

    // CSR of the off-diagonal pattern (both directions), neighbours ascending
    const double kk = double(kv) * double(kv);
    A.rowptr.assign(n0 + 1, 0);
    for (const Edge &e : E) { A.rowptr[e.a + 1]++; A.rowptr[e.b + 1]++; }
    for (int64_t p = 0; p < n0; ++p) A.rowptr[p + 1] += A.rowptr[p];
    const int64_t nnz = A.rowptr[n0];
    A.col.assign(nnz, 0);
    A.w.assign(nnz, 0.0);
    A.c_off.assign(nnz, 0.0);
    std::vector<int64_t> fill(A.rowptr.begin(), A.rowptr.end() - 1);
    for (const Edge &e : E) {   // E is sorted by (a, b): rows receive ascending columns
        int64_t ka = fill[e.a]++;
        A.col[ka] = int32_t(e.b); A.w[ka] = e.w; A.c_off[ka] = e.c / (kk * A.m[e.a]);
    }
    // second pass for the lower neighbours keeps columns ascending: insert then sort rows
    for (const Edge &e : E) {
        int64_t kb = fill[e.b]++;
        A.col[kb] = int32_t(e.a); A.w[kb] = e.w; A.c_off[kb] = e.c / (kk * A.m[e.b]);
    }
    std::vector<std::pair<int32_t, std::pair<double, double>>> row;
    A.wsum.assign(n0, 0.0);
    A.max_degree = 0;
    double rho = 0.0;
    for (int64_t p = 0; p < n0; ++p) {
        row.clear();
        for (int64_t k = A.rowptr[p]; k < A.rowptr[p + 1]; ++k) row.push_back({A.col[k], {A.w[k], A.c_off[k]}});
        std::sort(row.begin(), row.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        double ws = 0, wabs = 0;
        for (size_t i = 0; i < row.size(); ++i) {
            int64_t k = A.rowptr[p] + int64_t(i);
            A.col[k] = row[i].first; A.w[k] = row[i].second.first; A.c_off[k] = row[i].second.second;
            ws += A.w[k];
            wabs += std::fabs(A.w[k]);
        }
        A.wsum[p] = ws;
        A.max_degree = std::max<int32_t>(A.max_degree, int32_t(row.size()));
        // Gershgorin: spec(A) lies in the union of [A_pp - R_p, A_pp + R_p],
        // A_pp = sum_q w_pq / m_p, R_p = sum_q |w_pq| / m_p
        rho = std::max(rho, (ws + wabs) / A.m[p]);
    }
    // Gershgorin and the element bound are rigorous; the margin covers rounding
    A.rho_gershgorin = rho;
    A.rho_element = rho_elem;
    A.rho_rigorous = (1.0 + 1e-6) * std::min(rho, rho_elem);
    A.rho = A.rho_rigorous;
    A.rho_kind = DECBPM_RHO_RIGOROUS;
    if (d->spectral_bound == DECBPM_BOUND_DEFAULT || d->spectral_bound == DECBPM_BOUND_LANCZOS) {
        // The largest Ritz value theta of k Lanczos steps lies below lambda_max and
        // is typically within a fraction of a percent of it; 1.01 theta is then
        // checked per mesh (verify_upper_bound) before it replaces the rigorous bound.
        if (d->lanczos_steps < 0) return fail(DECBPM_ERR_INVALID_ARG, "lanczos_steps < 0");
        const int steps = d->lanczos_steps > 0 ? d->lanczos_steps : 200;
        const double theta = lanczos_lambda_max(A, steps);
        A.rho_lanczos = theta;
        if (theta > 0 && 1.01 * theta < A.rho_rigorous) {
            if (verify_upper_bound(A, 1.01 * theta, 128)) {
                A.rho = 1.01 * theta;
                A.rho_kind = DECBPM_RHO_LANCZOS_CHECKED;
            } else {
                A.rho_kind = DECBPM_RHO_LANCZOS_REJECTED;
            }
        }
    } else if (d->spectral_bound != DECBPM_BOUND_GERSHGORIN) {
        return fail(DECBPM_ERR_INVALID_ARG, "unknown spectral_bound %d", d->spectral_bound);
    }
    A.v.resize(n0); A.chib.resize(n0); A.c_diag.resize(n0);
    for (int64_t p = 0; p < n0; ++p) {
        A.v[p] = mV[p] / A.m[p];
        A.chib[p] = mchi[p] / A.m[p];
        A.c_diag[p] = cdiag[p] / (kk * A.m[p]);
    }

    if (d->ordering == DECBPM_ORDER_RCM) rcm(A.rowptr, A.col, n0, A.perm);
    else if (d->ordering == DECBPM_ORDER_DEFAULT || d->ordering == DECBPM_ORDER_HILBERT) hilbert_order(X, dim, n0, A.perm);
    else return fail(DECBPM_ERR_INVALID_ARG, "unknown ordering %d", d->ordering);
    A.iperm.assign(n0, 0);
    for (int64_t i = 0; i < n0; ++i) A.iperm[A.perm[i]] = int32_t(i);
    A.bandwidth = 0;
    for (const Edge &e : E) A.bandwidth = std::max<int64_t>(A.bandwidth, std::llabs(int64_t(A.iperm[e.a]) - A.iperm[e.b]));
    return DECBPM_OK;
}

void build_sell(const Assembly &a, Sell &s) {
    const int64_t n = a.n0;
    s.n_rows = n;
    s.n_slices = (n + kSlice - 1) / kSlice;
    s.slice_ptr.assign(s.n_slices + 1, 0);
    s.slice_w.assign(s.n_slices, 0);
    s.degree.assign(n, 0);
    for (int64_t r = 0; r < n; ++r) {
        const int32_t old = a.perm[r];
        s.degree[r] = int32_t(a.rowptr[old + 1] - a.rowptr[old]);
    }
    for (int64_t sl = 0; sl < s.n_slices; ++sl) {
        int32_t w = 0;
        for (int64_t r = sl * kSlice; r < std::min<int64_t>(n, (sl + 1) * kSlice); ++r) w = std::max(w, s.degree[r]);
        s.slice_w[sl] = w;
        s.slice_ptr[sl + 1] = s.slice_ptr[sl] + w * kSlice;
    }
    const int64_t total = s.slice_ptr[s.n_slices];
    s.col.assign(total, 0);
    s.w.assign(total, 0.0);
    s.c.assign(total, 0.0);
    std::vector<std::pair<int32_t, int64_t>> nb;
    for (int64_t sl = 0; sl < s.n_slices; ++sl) {
        for (int lane = 0; lane < kSlice; ++lane) {
            const int64_t r = sl * kSlice + lane;
            const int32_t self = r < n ? int32_t(r) : int32_t(sl * kSlice);
            nb.clear();
            if (r < n) {
                const int32_t old = a.perm[r];
                for (int64_t k = a.rowptr[old]; k < a.rowptr[old + 1]; ++k) nb.push_back({a.iperm[a.col[k]], k});
                std::sort(nb.begin(), nb.end());       // ascending internal column: better locality
            }
            for (int32_t j = 0; j < s.slice_w[sl]; ++j) {
                const int64_t idx = s.slice_ptr[sl] + int64_t(j) * kSlice + lane;
                if (j < int32_t(nb.size())) {
                    s.col[idx] = nb[j].first;
                    s.w[idx] = a.w[nb[j].second];
                    s.c[idx] = a.c_off[nb[j].second];
                } else {
                    s.col[idx] = self;
                }
            }
        }
    }
}

// Miller's backward recurrence J_{k-1} = (2k/a) J_k - J_{k+1}, normalized by
// J_0 + 2 sum_{k>=1} J_{2k} = 1.  Started far enough above max(kmax, a) that
// the arbitrary start values have decayed below double precision.
void bessel_sequence(double a, int kmax, double *J) {
    for (int k = 0; k <= kmax; ++k) J[k] = 0.0;
    if (a == 0.0) { J[0] = 1.0; return; }
    const int base = std::max(kmax, int(std::ceil(a)));
    const int start = 2 * ((base + 30 + int(std::sqrt(40.0 * base))) / 2) + 2;
    std::vector<double> Jall(start + 2, 0.0);
    double jp1 = 0.0, j = 1e-300, norm = 0.0;
    for (int k = start; k >= 1; --k) {
        const double jm1 = (2.0 * k / a) * j - jp1;
        jp1 = j;
        j = jm1;
        Jall[k - 1] = j;
        if (std::fabs(j) > 1e200) {                       // rescale to avoid overflow
            for (int q = k - 1; q <= start; ++q) Jall[q] *= 1e-200;
            j *= 1e-200; jp1 *= 1e-200;
        }
    }
    // J_start itself was the seed: Jall[start] unused; recompute normalization
    norm = Jall[0];
    for (int k = 2; k <= start; k += 2) norm += 2.0 * Jall[k];
    for (int k = 0; k <= kmax; ++k) J[k] = Jall[k] / norm;
}

void bessel_i_scaled(double a, double tol, std::vector<double> &s) {
    s.assign(1, 1.0);
    if (a <= 0.0) return;
    const int start = int(a + 40.0 + 12.0 * std::sqrt(a + 1.0));
    std::vector<double> v(start + 2, 0.0);
    double ip1 = 0.0, i = 1e-300;
    v[start] = i;
    for (int k = start; k >= 1; --k) {
        const double im1 = (2.0 * k / a) * i + ip1;
        ip1 = i;
        i = im1;
        v[k - 1] = i;
        if (i > 1e200) {                                   // rescale to avoid overflow
            for (int q = k - 1; q <= start; ++q) v[q] *= 1e-200;
            i *= 1e-200; ip1 *= 1e-200;
        }
    }
    double norm = v[0];
    for (int k = 1; k <= start; ++k) norm += 2.0 * v[k];
    int M = 0;
    for (int k = 0; k <= start; ++k)
        if (v[k] / norm >= tol * (v[0] / norm)) M = k;
    s.resize(M + 1);
    for (int k = 0; k <= M; ++k) s[k] = v[k] / norm;
}

int cheb_coefficients(const std::vector<double> &p, double rho, double h, double tol, Cheb &out) {
    using cd = std::complex<double>;
    const double c = 0.5 * rho, r = 0.5 * rho;
    if (tol <= 0) tol = 1e-16;
    out = Cheb();
    if (p.size() == 1) {
        // exp(-i h p1 lambda) = exp(-i h p1 c) exp(-i (h p1 r) x)
        const double a = h * p[0] * r;
        const double aa = std::fabs(a);
        int kmax = int(aa + 40 + 12 * std::cbrt(aa + 1.0));
        std::vector<double> J(kmax + 1);
        bessel_sequence(aa, kmax, J.data());
        // smallest M with tail 2 sum_{k>M} |J_k| <= tol
        std::vector<double> tail(kmax + 2, 0.0);
        for (int k = kmax; k >= 0; --k) tail[k] = tail[k + 1] + 2.0 * std::fabs(J[k]);
        int M = 0;
        while (M < kmax && tail[M + 1] > tol) ++M;
        M = std::max(M, 2);
        out.M = M;
        out.theta0 = -h * p[0] * c;
        out.f0 = std::exp(cd(0.0, h * p[0] * c));
        out.a.resize(M + 1);
        for (int k = 0; k <= M; ++k) {
            // (-i)^k J_k(a) is purely real or imaginary; J_k(-a) = (-1)^k J_k(a)
            const double jk = J[k] * ((a < 0 && (k & 1)) ? -1.0 : 1.0) * (k == 0 ? 1.0 : 2.0);
            switch (k & 3) {
                case 0: out.a[k] = cd(jk, 0.0); break;
                case 1: out.a[k] = cd(0.0, -jk); break;
                case 2: out.a[k] = cd(-jk, 0.0); break;
                default: out.a[k] = cd(0.0, jk); break;
            }
        }
        return DECBPM_OK;
    }
    // general p_n: coefficients by a discrete cosine transform of f at
    // Chebyshev points; the number of points exceeds twice the degree that the
    // phase range of f demands, so aliasing stays below double precision.
    double slope = 0.0, lam = rho;
    for (size_t n = 1; n <= p.size(); ++n) slope += double(n) * std::fabs(p[n - 1]) * std::pow(lam, double(n - 1));
    const double est = std::fabs(h) * r * slope;
    if (est > 2e6) return fail(DECBPM_ERR_UNSUPPORTED, "Chebyshev degree estimate %.3g too large (reduce dz)", est);
    int N = 64;
    while (N < 2 * int(est + 64)) N *= 2;
    std::vector<cd> f(N);
    const double pi = std::acos(-1.0);
    auto gfun = [&](double l) {
        double g = 0.0, pw = 1.0;
        for (size_t n = 1; n <= p.size(); ++n) { pw *= -l; g += p[n - 1] * pw; }
        return g;
    };
    const double gc = gfun(c);
    out.theta0 = h * gc;
    out.f0 = std::exp(cd(0.0, h * (gfun(0.0) - gc)));
    for (int j = 0; j < N; ++j) {
        const double x = std::cos(pi * (j + 0.5) / N);
        f[j] = std::exp(cd(0.0, h * (gfun(c + r * x) - gc)));
    }
    // cos(pi k (j + 1/2) / N) = cos(pi m / (2N)), m = k (2j + 1) mod 4N: the
    // angle is reduced exactly in integers and then by the symmetries of the
    // cosine to [0, pi/4], so every table value is correct to about an ulp (a
    // rounded argument pi k (j + 1/2) / N of up to ~pi N radians would put
    // noise of ~1e-15 into every coefficient).  Sums are compensated
    // (Neumaier), so the coefficients carry noise of ~2 eps / sqrt(N) only.
    const int64_t n4 = 4 * int64_t(N), n2 = 2 * int64_t(N);
    auto cq = [&](int64_t m) {
        m %= n4;
        if (m > n2) m = n4 - m;                       // cos(2 pi - t) = cos t
        double sg = 1.0;
        if (m > N) { m = n2 - m; sg = -1.0; }         // cos(pi - t) = -cos t
        return m <= N / 2 ? sg * std::cos(pi * double(m) / double(n2)) : sg * std::sin(pi * double(N - m) / double(n2));
    };
    std::vector<double> ctab(n4);
    for (int64_t m = 0; m < n4; ++m) ctab[m] = cq(m);
    auto neumaier = [](double &sum, double &comp, double x) {
        const double t = sum + x;
        comp += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
        sum = t;
    };
    std::vector<cd> a(N);
    for (int k = 0; k < N; ++k) {
        double sr = 0, cr = 0, si = 0, ci = 0;
        for (int j = 0; j < N; ++j) {
            const double cs = ctab[(int64_t(k) * (2 * j + 1)) % n4];
            neumaier(sr, cr, f[j].real() * cs);
            neumaier(si, ci, f[j].imag() * cs);
        }
        a[k] = cd(sr + cr, si + ci) * ((k == 0 ? 1.0 : 2.0) / N);
    }
    // truncation: coefficients below the noise level eta of the transform do
    // not count towards the tail (their sum over N terms would otherwise keep
    // the degree near N)
    const double floor_tol = std::max(tol, 1e-15);
    const double eta = 16.0 * 2.220446049250313e-16 / std::sqrt(double(N));
    std::vector<double> tail(N + 1, 0.0);
    for (int k = N - 1; k >= 0; --k) tail[k] = tail[k + 1] + std::max(std::abs(a[k]) - eta, 0.0);
    int M = 0;
    while (M < N - 1 && tail[M + 1] > floor_tol) ++M;
    M = std::max(M, 2);
    out.M = M;
    out.a.assign(a.begin(), a.begin() + M + 1);
    return DECBPM_OK;
}

}  // namespace decbpm
