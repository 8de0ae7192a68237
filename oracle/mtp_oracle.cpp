// Oracle: plain FP64 CPU evaluation of the Moment Tensor Potential (Sec. 2.1, Eqs. 1-6).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference that the
// CUDA path is checked against.  It shares no code, header or table with the CUDA path and
// is never linked into the product library; only tests/, __graft_entry__.smoke() and
// bench.py's CPU-baseline leg load it (through oracle/__init__.py).
//
// Every quantity is computed from its definition, in the paper's order:
//   neighbourhood   n_i = {(z_j, r_ij) : |r_ij| < R_cut}, r_ij from atom i to atom j   (Eq. 1)
//   radial basis    Q_b(r) = T_{b-1}(x) (R_cut - r)^2 for r < R_cut, else 0             (Eq. 4)
//                   x = (2r - R_min - R_cut) / (R_cut - R_min) maps [R_min, R_cut] to [-1, 1]
//   radial funcs    f_mu(r, z_i, z_j) = sum_b c[z_i][z_j][mu][b] Q_b(r)                  (Eq. 3)
//   moments         M_{mu,nu} = sum_j f_mu(|r_ij|) r_ij (x) ... (x) r_ij  (nu factors)    (Sec. 2.1)
//   basis           every connected contraction is the sum over all index values of its
//                   edges of the product of its moment entries; a basis function is the
//                   product of its connected contractions                              (Eqs. 5-6)
//   site energy     V_i = sum_a xi_a B_a(n_i)                                             (Eq. 2)
//   energy          E = sum_i V_i                                                         (Eq. 1)
//   forces          F_k = -dE/dx_k, by the chain rule through every step above
//   virial          W = -dE/d(eps) for a homogeneous strain x -> (I + eps) x of cell and atoms
//
// The scalar type is a template parameter.  With Dual (value + one tangent) the same code
// returns the exact derivative of E, F and W along one direction of the parameters
// theta = {xi, c}; that is how the oracle differentiates the training loss (Eqs. 7, 11, 12).
//
// A moment entry is addressed by (mu, a, b, c): the tensor entry whose index tuple holds
// a x's, b y's and c z's (nu = a + b + c).  All index tuples with the same counts hold the
// same value because the tensor is symmetric, so this is just the definition written out.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <array>
#include <algorithm>
#include <tuple>
#include <functional>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double x) : v(x), d(0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
inline double tan_(double) { return 0.0; }
inline double tan_(Dual x) { return x.d; }

// ------------------------------------------------------------------------------------------
// Basis description (parsed from the level table written by oracle/levels.py)
// ------------------------------------------------------------------------------------------
struct Component {
    std::vector<int> mu, nu;                 // node labels
    std::vector<std::pair<int, int>> edges;  // one entry per contracted index pair
};

struct Model {
    int L = 0, S = 0, NQ = 0, Nmu = 0, numax = 0, m = 0;
    double rmin = 0, rcut = 0;
    std::vector<Component> comps;            // distinct connected components
    std::vector<std::vector<int>> basis;     // basis function -> component ids (with repeats)
};

// ------------------------------------------------------------------------------------------
// Neighbourhoods (Eq. 1): every (j, s) with |x_j + s H - x_i| < R_cut, excluding (i, s = 0).
// ------------------------------------------------------------------------------------------
struct Pair {
    int j;
    int s[3];
    double d[3];  // r_ij = x_j + s H - x_i
};

// displacement written in one fixed operation order: shift first, then x_j + shift - x_i
inline void displacement(const double* xi, const double* xj, const double* H, const int* s, double* d) {
    for (int k = 0; k < 3; ++k) {
        double sh = (double)s[0] * H[0 * 3 + k];
        sh = sh + (double)s[1] * H[1 * 3 + k];
        sh = sh + (double)s[2] * H[2 * 3 + k];
        d[k] = (xj[k] + sh) - xi[k];
    }
}

inline double norm2(const double* d) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

void inverse3(const double* H, double* Hi, double* vol) {
    double a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7], k = H[8];
    double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
    Hi[0] = (e * k - f * h) / det; Hi[1] = (c * h - b * k) / det; Hi[2] = (b * f - c * e) / det;
    Hi[3] = (f * g - d * k) / det; Hi[4] = (a * k - c * g) / det; Hi[5] = (c * d - a * f) / det;
    Hi[6] = (d * h - e * g) / det; Hi[7] = (b * g - a * h) / det; Hi[8] = (a * e - b * d) / det;
    *vol = std::fabs(det);
}

// Perpendicular width of the cell along lattice direction k: volume / |a_l x a_m|.
void widths(const double* H, double* w) {
    double Hi[9], vol;
    inverse3(H, Hi, &vol);
    for (int k = 0; k < 3; ++k) {
        const double* a = H + ((k + 1) % 3) * 3;
        const double* b = H + ((k + 2) % 3) * 3;
        double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
        w[k] = vol / std::sqrt(cx * cx + cy * cy + cz * cz);
    }
}

// Brute force over every atom j and every image shift that could lie within R_cut:
// |(f_j - f_i + s)_k| * width_k <= |r| bounds each shift component from the fractional
// displacement f, so the finite range below (rounded outwards) contains every solution.
// With `cand` (ascending atom indices) only those atoms are tried as j: the result is the full
// list whenever every neighbour of i is among them.
std::vector<Pair> neighbours_of(int i, int n, const double* pos, const double* H, double rcut,
                                const std::vector<int>* cand = nullptr) {
    double Hi[9], vol, w[3];
    inverse3(H, Hi, &vol);
    widths(H, w);
    const double rc2 = rcut * rcut;
    std::vector<Pair> out;
    const int count = cand ? (int)cand->size() : n;
    for (int t = 0; t < count; ++t) {
        const int j = cand ? (*cand)[t] : t;
        double dx[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
        int lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            double f = dx[0] * Hi[0 * 3 + k] + dx[1] * Hi[1 * 3 + k] + dx[2] * Hi[2 * 3 + k];
            double reach = rcut / w[k];
            lo[k] = (int)std::floor(-f - reach);
            hi[k] = (int)std::ceil(-f + reach);
        }
        int s[3];
        for (s[0] = lo[0]; s[0] <= hi[0]; ++s[0])
            for (s[1] = lo[1]; s[1] <= hi[1]; ++s[1])
                for (s[2] = lo[2]; s[2] <= hi[2]; ++s[2]) {
                    if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
                    Pair p;
                    p.j = j;
                    std::memcpy(p.s, s, sizeof s);
                    displacement(pos + 3 * i, pos + 3 * j, H, s, p.d);
                    if (norm2(p.d) < rc2) out.push_back(p);
                }
    }
    std::sort(out.begin(), out.end(), [](const Pair& a, const Pair& b) {
        return std::make_tuple(a.j, a.s[0], a.s[1], a.s[2]) < std::make_tuple(b.j, b.s[0], b.s[1], b.s[2]);
    });
    return out;
}

// ------------------------------------------------------------------------------------------
// Radial part (Eqs. 3-4)
// ------------------------------------------------------------------------------------------
// Q_b and dQ_b/dr for b = 1..NQ, r < R_cut.
void radial_basis(const Model& M, double r, std::vector<double>& Q, std::vector<double>& dQ) {
    const double span = M.rcut - M.rmin;
    const double x = (2.0 * r - M.rmin - M.rcut) / span;
    const double dxdr = 2.0 / span;
    std::vector<double> T(M.NQ), dT(M.NQ);
    for (int k = 0; k < M.NQ; ++k) {
        if (k == 0) { T[k] = 1.0; dT[k] = 0.0; }
        else if (k == 1) { T[k] = x; dT[k] = 1.0; }
        else {
            T[k] = 2.0 * x * T[k - 1] - T[k - 2];
            dT[k] = 2.0 * T[k - 1] + 2.0 * x * dT[k - 1] - dT[k - 2];
        }
    }
    const double u = M.rcut - r;
    Q.resize(M.NQ);
    dQ.resize(M.NQ);
    for (int k = 0; k < M.NQ; ++k) {
        Q[k] = T[k] * u * u;
        dQ[k] = dT[k] * dxdr * u * u - 2.0 * T[k] * u;
    }
}

// ------------------------------------------------------------------------------------------
// Moments and contractions
// ------------------------------------------------------------------------------------------
inline int midx(const Model& M, int mu, int a, int b, int c) {
    const int D = M.numax + 1;
    return ((mu * D + a) * D + b) * D + c;
}
inline int msize(const Model& M) {
    const int D = M.numax + 1;
    return M.Nmu * D * D * D;
}

inline double ipow(double x, int k) {
    double r = 1.0;
    for (int t = 0; t < k; ++t) r *= x;
    return r;
}

// Value of one connected contraction: sum over every assignment of {x,y,z} to its edges of
// the product of the node entries that the assignment selects.
template <class T>
T component_value(const Model& M, const Component& C, const std::vector<T>& mom) {
    const int n = (int)C.mu.size();
    const int E = (int)C.edges.size();
    if (E == 0) return mom[midx(M, C.mu[0], 0, 0, 0)];
    std::vector<int> idx(E, 0);
    std::vector<std::array<int, 3>> cnt(n);
    T total = 0.0;
    while (true) {
        for (auto& q : cnt) q = {0, 0, 0};
        for (int e = 0; e < E; ++e) {
            cnt[C.edges[e].first][idx[e]]++;
            cnt[C.edges[e].second][idx[e]]++;
        }
        T prod = 1.0;
        for (int u = 0; u < n; ++u) prod = prod * mom[midx(M, C.mu[u], cnt[u][0], cnt[u][1], cnt[u][2])];
        total += prod;
        int e = 0;
        while (e < E && ++idx[e] == 3) idx[e++] = 0;
        if (e == E) break;
    }
    return total;
}

// Adds  w * d(component value)/d(moment entry)  to dmom, by the product rule over the nodes.
template <class T>
void component_grad(const Model& M, const Component& C, const std::vector<T>& mom, T w, std::vector<T>& dmom) {
    const int n = (int)C.mu.size();
    const int E = (int)C.edges.size();
    if (E == 0) { dmom[midx(M, C.mu[0], 0, 0, 0)] += w; return; }
    std::vector<int> idx(E, 0);
    std::vector<std::array<int, 3>> cnt(n);
    while (true) {
        for (auto& q : cnt) q = {0, 0, 0};
        for (int e = 0; e < E; ++e) {
            cnt[C.edges[e].first][idx[e]]++;
            cnt[C.edges[e].second][idx[e]]++;
        }
        for (int u = 0; u < n; ++u) {
            T prod = w;
            for (int v = 0; v < n; ++v)
                if (v != u) prod = prod * mom[midx(M, C.mu[v], cnt[v][0], cnt[v][1], cnt[v][2])];
            dmom[midx(M, C.mu[u], cnt[u][0], cnt[u][1], cnt[u][2])] += prod;
        }
        int e = 0;
        while (e < E && ++idx[e] == 3) idx[e++] = 0;
        if (e == E) break;
    }
}

// One neighbourhood: V_i, the basis values B_a and dV_i/dr_ij for every neighbour.
template <class T>
struct Site {
    T V;
    std::vector<T> B;
    std::vector<std::array<T, 3>> g;
};

template <class T>
Site<T> eval_site(const Model& M, const std::vector<T>& xi, const std::vector<T>& c, int zi,
                  const std::vector<Pair>& nb, const int* types) {
    const int P = (int)nb.size();
    // radial functions f_mu and their r-derivatives for every pair (Eq. 3)
    std::vector<std::vector<T>> f(P, std::vector<T>(M.Nmu)), df(P, std::vector<T>(M.Nmu));
    std::vector<double> r(P);
    std::vector<double> Q, dQ;
    for (int p = 0; p < P; ++p) {
        r[p] = std::sqrt(norm2(nb[p].d));
        radial_basis(M, r[p], Q, dQ);
        const int zj = types[nb[p].j];
        for (int mu = 0; mu < M.Nmu; ++mu) {
            T s = 0.0, ds = 0.0;
            for (int b = 0; b < M.NQ; ++b) {
                const T cc = c[((zi * M.S + zj) * M.Nmu + mu) * M.NQ + b];
                s += cc * Q[b];
                ds += cc * dQ[b];
            }
            f[p][mu] = s;
            df[p][mu] = ds;
        }
    }
    // moments: entry (mu, a, b, c) = sum_j f_mu x^a y^b z^c
    std::vector<T> mom(msize(M), T(0.0));
    for (int p = 0; p < P; ++p)
        for (int mu = 0; mu < M.Nmu; ++mu)
            for (int a = 0; a <= M.numax; ++a)
                for (int b = 0; a + b <= M.numax; ++b)
                    for (int cc = 0; a + b + cc <= M.numax; ++cc)
                        mom[midx(M, mu, a, b, cc)] +=
                            f[p][mu] * (ipow(nb[p].d[0], a) * ipow(nb[p].d[1], b) * ipow(nb[p].d[2], cc));
    // connected contractions, then basis functions as their products (Eq. 2)
    std::vector<T> cv(M.comps.size());
    for (size_t k = 0; k < M.comps.size(); ++k) cv[k] = component_value(M, M.comps[k], mom);
    Site<T> out;
    out.V = 0.0;
    out.B.resize(M.m);
    for (int a = 0; a < M.m; ++a) {
        T prod = 1.0;
        for (int k : M.basis[a]) prod = prod * cv[k];
        out.B[a] = prod;
        out.V += xi[a] * prod;
    }
    // dV/d(component value): product rule over the factors of each basis function
    std::vector<T> dcv(M.comps.size(), T(0.0));
    for (int a = 0; a < M.m; ++a) {
        const auto& fac = M.basis[a];
        for (size_t t = 0; t < fac.size(); ++t) {
            T prod = xi[a];
            for (size_t u = 0; u < fac.size(); ++u)
                if (u != t) prod = prod * cv[fac[u]];
            dcv[fac[t]] += prod;
        }
    }
    std::vector<T> dmom(msize(M), T(0.0));
    for (size_t k = 0; k < M.comps.size(); ++k) component_grad(M, M.comps[k], mom, dcv[k], dmom);
    // dV/dr_ij = sum over entries of dV/dM * d(f_mu(r) x^a y^b z^c)/dr_ij
    out.g.assign(P, {T(0.0), T(0.0), T(0.0)});
    for (int p = 0; p < P; ++p) {
        const double* d = nb[p].d;
        const double rhat[3] = {d[0] / r[p], d[1] / r[p], d[2] / r[p]};
        for (int mu = 0; mu < M.Nmu; ++mu)
            for (int a = 0; a <= M.numax; ++a)
                for (int b = 0; a + b <= M.numax; ++b)
                    for (int cc = 0; a + b + cc <= M.numax; ++cc) {
                        const T w = dmom[midx(M, mu, a, b, cc)];
                        if (val(w) == 0.0 && tan_(w) == 0.0) continue;
                        const double mono = ipow(d[0], a) * ipow(d[1], b) * ipow(d[2], cc);
                        const double gx = a ? a * ipow(d[0], a - 1) * ipow(d[1], b) * ipow(d[2], cc) : 0.0;
                        const double gy = b ? b * ipow(d[0], a) * ipow(d[1], b - 1) * ipow(d[2], cc) : 0.0;
                        const double gz = cc ? cc * ipow(d[0], a) * ipow(d[1], b) * ipow(d[2], cc - 1) : 0.0;
                        const double grad[3] = {gx, gy, gz};
                        for (int k = 0; k < 3; ++k)
                            out.g[p][k] += w * (df[p][mu] * (rhat[k] * mono) + f[p][mu] * grad[k]);
                    }
    }
    return out;
}

Model* parse_model(int L, int S, int NQ, double rmin, double rcut, const int* tab, int len) {
    Model* M = new Model;
    M->L = L; M->S = S; M->NQ = NQ; M->rmin = rmin; M->rcut = rcut;
    int pos = 0;
    M->m = tab[pos++];
    std::vector<std::vector<int>> codes;
    int maxmu = 0, maxnu = 0;
    for (int a = 0; a < M->m; ++a) {
        pos++;  // level
        const int ncomp = tab[pos++];
        std::vector<int> ids;
        for (int t = 0; t < ncomp; ++t) {
            const int n = tab[pos];
            const int clen = 1 + 2 * n + n * (n - 1) / 2;
            std::vector<int> code(tab + pos, tab + pos + clen);
            pos += clen;
            int id = -1;
            for (size_t q = 0; q < codes.size(); ++q)
                if (codes[q] == code) id = (int)q;
            if (id < 0) {
                id = (int)codes.size();
                codes.push_back(code);
                Component C;
                for (int u = 0; u < n; ++u) {
                    C.mu.push_back(code[1 + 2 * u]);
                    C.nu.push_back(code[2 + 2 * u]);
                    maxmu = std::max(maxmu, code[1 + 2 * u]);
                    maxnu = std::max(maxnu, code[2 + 2 * u]);
                }
                int q = 1 + 2 * n;
                for (int u = 0; u < n; ++u)
                    for (int v = u + 1; v < n; ++v) {
                        for (int e = 0; e < code[q]; ++e) C.edges.push_back({u, v});
                        ++q;
                    }
                M->comps.push_back(C);
            }
            ids.push_back(id);
        }
        M->basis.push_back(ids);
    }
    M->Nmu = maxmu + 1;
    M->numax = maxnu;
    return M;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C interface used by oracle/__init__.py (ctypes)
// ------------------------------------------------------------------------------------------
extern "C" {

void* oracle_model_create(int L, int S, int NQ, double rmin, double rcut, const int* table, int len) {
    return parse_model(L, S, NQ, rmin, rcut, table, len);
}
void oracle_model_free(void* p) { delete (Model*)p; }
int oracle_model_nmu(void* p) { return ((Model*)p)->Nmu; }
int oracle_model_m(void* p) { return ((Model*)p)->m; }

// Q_b(r) and dQ_b/dr, b = 1..NQ, for pinning the radial basis of Eq. 4 in isolation.
void oracle_radial(void* p, double r, double* Q, double* dQ) {
    std::vector<double> q, dq;
    radial_basis(*(Model*)p, r, q, dq);
    for (size_t k = 0; k < q.size(); ++k) { Q[k] = q[k]; dQ[k] = dq[k]; }
}

// Neighbour lists of the atoms listed in `which` (all atoms when which == NULL, count = n).
// Writes counts[count]; when the output arrays are non-NULL (capacity cap pairs) also the
// pairs in canonical order (j, s) per atom, concatenated.  Returns the total pair count, or
// -1 if cap is too small.
long oracle_neighbors(int n, const double* pos, const double* cell, double rcut, const int* which, int count,
                      int* counts, int* nbr_j, int* nbr_s, double* nbr_d, long cap) {
    std::vector<std::vector<Pair>> all(count);
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < count; ++t) all[t] = neighbours_of(which ? which[t] : t, n, pos, cell, rcut);
    long total = 0;
    for (int t = 0; t < count; ++t) {
        counts[t] = (int)all[t].size();
        total += (long)all[t].size();
    }
    if (!nbr_j) return total;
    if (total > cap) return -1;
    long q = 0;
    for (int t = 0; t < count; ++t)
        for (const Pair& p : all[t]) {
            nbr_j[q] = p.j;
            for (int k = 0; k < 3; ++k) {
                if (nbr_s) nbr_s[3 * q + k] = p.s[k];
                if (nbr_d) nbr_d[3 * q + k] = p.d[k];
            }
            ++q;
        }
    return total;
}

// Energy, forces and virial of one periodic configuration.
//   xi[m], c[S*S*Nmu*NQ]; tangents dxi/dc may be NULL (then derivative outputs are skipped).
//   forces[n*3], virial[9] (row-major W_ab = -sum g_a r_b), site[n] and batoms[n*m] may be NULL.
//   d_energy, d_forces[n*3], d_virial[9]: derivatives along (dxi, dc) when tangents given.
int oracle_eval(void* model, const double* xi_, const double* c_, int n, const double* pos, const int* types,
                const double* cell, double* energy, double* forces, double* virial, double* site,
                double* batoms, const double* dxi, const double* dc, double* d_energy, double* d_forces,
                double* d_virial, int nthreads) {
    const Model& M = *(Model*)model;
    const int nc = M.S * M.S * M.Nmu * M.NQ;
    for (int i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= M.S) return 1;
    const bool tangent = dxi && dc;
    std::vector<Dual> xi(M.m), c(nc);
    for (int a = 0; a < M.m; ++a) xi[a] = Dual(xi_[a], tangent ? dxi[a] : 0.0);
    for (int k = 0; k < nc; ++k) c[k] = Dual(c_[k], tangent ? dc[k] : 0.0);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    std::vector<Site<Dual>> sites(n);
    std::vector<std::vector<Pair>> nbrs(n);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i) {
        nbrs[i] = neighbours_of(i, n, pos, cell, M.rcut);
        sites[i] = eval_site(M, xi, c, types[i], nbrs[i], types);
    }
    Dual E = 0.0;
    std::vector<Dual> F(3 * n, Dual(0.0)), W(9, Dual(0.0));
    for (int i = 0; i < n; ++i) {
        E += sites[i].V;
        for (size_t p = 0; p < nbrs[i].size(); ++p) {
            const Pair& pr = nbrs[i][p];
            for (int a = 0; a < 3; ++a) {
                F[3 * i + a] += sites[i].g[p][a];     // F_i = -dE/dx_i, dr_ij/dx_i = -1
                F[3 * pr.j + a] -= sites[i].g[p][a];  // F_j = -dE/dx_j, dr_ij/dx_j = +1
                for (int b = 0; b < 3; ++b) W[3 * a + b] -= sites[i].g[p][a] * pr.d[b];
            }
        }
    }
    if (energy) *energy = E.v;
    if (d_energy) *d_energy = E.d;
    for (int k = 0; k < 3 * n; ++k) {
        if (forces) forces[k] = F[k].v;
        if (d_forces) d_forces[k] = F[k].d;
    }
    for (int k = 0; k < 9; ++k) {
        if (virial) virial[k] = W[k].v;
        if (d_virial) d_virial[k] = W[k].d;
    }
    for (int i = 0; i < n; ++i) {
        if (site) site[i] = sites[i].V.v;
        if (batoms)
            for (int a = 0; a < M.m; ++a) batoms[(long)i * M.m + a] = sites[i].B[a].v;
    }
    return 0;
}

// Site energies, basis rows and forces restricted to a sample of atoms of a large
// configuration: V_i and B(n_i) for i in `which`, and the force on each sampled atom k,
//   F_k = -dE/dx_k = sum over pairs (k, j, s) of n_k with j != k of dV_k/dr_kj
//                    - sum over atoms i != k of sum over pairs (i, k, s) of n_i of dV_i/dr_ik.
// A self-image pair (k, k, s != 0) has r = s H, which does not move with x_k, so it gives no
// force (in the full evaluation its two terms cancel).  Every i with k in n_i is within R_cut of
// k, and each of i's neighbours is within 2 R_cut of k, so the neighbour lists are searched only
// among the atoms that have an image within 2 R_cut of k (the same lists as a search over all atoms).
int oracle_eval_sampled(void* model, const double* xi_, const double* c_, int n, const double* pos,
                        const int* types, const double* cell, const int* which, int count, double* site,
                        double* batoms, double* forces, int nthreads) {
    const Model& M = *(Model*)model;
    const int nc = M.S * M.S * M.Nmu * M.NQ;
    for (int t = 0; t < count; ++t)
        if (which[t] < 0 || which[t] >= n) return 1;
    for (int i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= M.S) return 1;
    std::vector<double> xi(xi_, xi_ + M.m), c(c_, c_ + nc);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < count; ++t) {
        const int k = which[t];
        std::vector<int> cand;
        for (const Pair& p : neighbours_of(k, n, pos, cell, 2.0 * M.rcut)) cand.push_back(p.j);
        cand.push_back(k);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        std::vector<Pair> nk = neighbours_of(k, n, pos, cell, M.rcut, &cand);
        Site<double> sk = eval_site(M, xi, c, types[k], nk, types);
        if (site) site[t] = sk.V;
        if (batoms)
            for (int a = 0; a < M.m; ++a) batoms[(long)t * M.m + a] = sk.B[a];
        if (!forces) continue;
        double F[3] = {0, 0, 0};
        for (size_t p = 0; p < nk.size(); ++p)
            if (nk[p].j != k)
                for (int a = 0; a < 3; ++a) F[a] += sk.g[p][a];
        // contributions of V_i for each distinct neighbour atom i != k
        std::vector<int> others;
        for (const Pair& p : nk)
            if (p.j != k) others.push_back(p.j);
        std::sort(others.begin(), others.end());
        others.erase(std::unique(others.begin(), others.end()), others.end());
        for (int i : others) {
            std::vector<Pair> ni = neighbours_of(i, n, pos, cell, M.rcut, &cand);
            Site<double> si = eval_site(M, xi, c, types[i], ni, types);
            for (size_t p = 0; p < ni.size(); ++p)
                if (ni[p].j == k)
                    for (int a = 0; a < 3; ++a) F[a] -= si.g[p][a];
        }
        for (int a = 0; a < 3; ++a) forces[3 * t + a] = F[a];
    }
    return 0;
}

}  // extern "C"
