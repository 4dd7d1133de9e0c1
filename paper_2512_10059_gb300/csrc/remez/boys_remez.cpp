// Rational minimax (Remez) generator for the FP32 tier of libboys.
//
// Host-only C++ in extended precision (`long double`: 64-bit significand on
// x86-64, binary128 on AArch64).  For every kmax in [0, 32] it
//   * sets x0(kmax) by Eq. x0 and x1(kmax) by solving Eq. x1 for the region-C
//     budget,
//   * fits r_{A,kmax} ~ F_kmax on [0, x0) with the weight rho_{A,kmax}
//     (Eq. rhoAk) and r_B ~ F_0 on [x0, x1) with weight 1,
//   * picks each approximant from the Walsh table as in Section II.D: the
//     first anti-diagonal n+m = d on which some (n, m) reaches the target
//     error, and on it the one with the smallest error,
//   * rounds the coefficients to FP32 and verifies the whole FP32 evaluation
//     (Algorithm 1 in float arithmetic, the kernel's operation order) against
//     extended-precision reference values on a dense grid, tightening the
//     target and refitting if the end-to-end error exceeds its budget,
// and writes a C header of FP32 tables.
//
// The Remez iteration follows the six steps of Section II.B:
//   1. initial equioscillation nodes (Chebyshev-distributed; randomly
//      perturbed restarts if no pole-free solution exists; for strongly
//      weighted problems, continuation from the unweighted problem through
//      rho^s, s = 0, 1/4, ..., 1),
//   2. solve rho (f - p/q)(x_i) = (-1)^i E at fixed nodes: functionals built
//      from the nodes' divided-difference weights annihilate p, and a basis
//      orthonormal in the weighted discrete inner product sum |w_i|/rho_i g h
//      turns the remaining equations for q into a real symmetric eigenvalue
//      problem (solved by cyclic Jacobi) with m+1 solutions (q_j, E_j),
//   3. keep the solution whose q has no zero in the interval (Sturm sequence),
//   4. stop when max |rho (f - r)| - |E| is small relative to |E|,
//   5. move the nodes to alternating local maxima of |rho (f - r)| found on a
//      grid and refined by golden-section search, keeping the global maximum,
//   6. abort when the smallest error at the new alternating nodes already
//      exceeds the target (de la Vallee-Poussin: no (n, m) approximant can do
//      better).
// Reference values come from the all-positive series of the reference-values
// section (F_k = e^{-x}/2 sum_l x^l / prod_{j<=l}(k+j+1/2)).
//
// Usage: boys_remez > boys_coeffs_fp32.h   (progress and the verification
// report go to stderr).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

typedef long double real;
typedef std::vector<real> vec;

static const real PI_L = 3.141592653589793238462643383279502884L;

// ------------------------------------------------------------- reference F_k

static real boys_ref(int k, real x) {
    real kh = k + 0.5L;
    real t = 1.0L / kh, s = t;
    for (int l = 0; l < 100000; ++l) {
        real q = x / (kh + (real)(l + 1));
        if (q < 1.0L && t * q / (1.0L - q) <= 1e-24L * s) break;
        t *= q;
        s += t;
    }
    return 0.5L * expl(-x) * s;
}

// rho_{A,k}(x) = max_l prod_{n=l}^{k-1} x / (n + 1/2)   (Eq. rhoAk, zeroth order)
static real rho_A(int k, real x) {
    real best = 1.0L, prod = 1.0L;
    for (int n = k - 1; n >= 0; --n) {
        prod *= x / (n + 0.5L);
        best = std::max(best, prod);
    }
    return best;
}

// x0 = max{1, (prod_{k<kmax} (k+1/2))^{1/kmax}}   (Eq. x0)
static real x0_of(int kmax) {
    if (kmax == 0) return 1.0L;
    real lp = 0.0L;
    for (int k = 0; k < kmax; ++k) lp += logl(k + 0.5L);
    return std::max(1.0L, expl(lp / kmax));
}

// asymptotic-form error Gamma(k+1/2, x) / (2 x^{k+1/2}) = Gamma(k+1/2)/(2x^{k+1/2}) - F_k(x)
static real asym_err(int k, real x) {
    return expl(lgammal(k + 0.5L) - (k + 0.5L) * logl(x)) / 2.0L - boys_ref(k, x);
}

// x1 solves asym_err(kmax, x1) = eps (Eq. x1); the error decreases in x.
static real x1_of(int kmax, real eps) {
    real lo = 0.5L, hi = 200.0L;
    for (int it = 0; it < 200; ++it) {
        real mid = 0.5L * (lo + hi);
        if (asym_err(kmax, mid) > eps) lo = mid; else hi = mid;
    }
    return hi;
}

// ------------------------------------------------------------- small linear algebra

// Cyclic Jacobi for a symmetric matrix a (n x n, row-major): eigenvalues in d,
// eigenvectors in columns of v.
static void jacobi(int n, vec a, vec& d, vec& v) {
    v.assign(n * n, 0.0L);
    for (int i = 0; i < n; ++i) v[i * n + i] = 1.0L;
    for (int sweep = 0; sweep < 100; ++sweep) {
        real off = 0.0L;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
        if (off < 1e-36L) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                real apq = a[p * n + q];
                if (fabsl(apq) < 1e-300L) continue;
                real theta = (a[q * n + q] - a[p * n + p]) / (2.0L * apq);
                real t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
                real c = 1.0L / sqrtl(t * t + 1.0L), s = t * c;
                for (int r = 0; r < n; ++r) {
                    real arp = a[r * n + p], arq = a[r * n + q];
                    a[r * n + p] = c * arp - s * arq;
                    a[r * n + q] = s * arp + c * arq;
                }
                for (int r = 0; r < n; ++r) {
                    real apr = a[p * n + r], aqr = a[q * n + r];
                    a[p * n + r] = c * apr - s * aqr;
                    a[q * n + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < n; ++r) {
                    real vrp = v[r * n + p], vrq = v[r * n + q];
                    v[r * n + p] = c * vrp - s * vrq;
                    v[r * n + q] = s * vrp + c * vrq;
                }
            }
    }
    d.resize(n);
    for (int i = 0; i < n; ++i) d[i] = a[i * n + i];
}

// Polynomials are coefficient vectors in the scaled variable t, lowest degree first.
static real peval(const vec& c, real t) {
    real v = 0.0L;
    for (int i = (int)c.size() - 1; i >= 0; --i) v = v * t + c[i];
    return v;
}

static vec pderiv(const vec& c) {
    vec d;
    for (size_t i = 1; i < c.size(); ++i) d.push_back(c[i] * (real)i);
    if (d.empty()) d.push_back(0.0L);
    return d;
}

static void ptrim(vec& c) {
    real mx = 0.0L;
    for (real v : c) mx = std::max(mx, fabsl(v));
    while (c.size() > 1 && fabsl(c.back()) <= 1e-30L * mx) c.pop_back();
}

// remainder of a / b (b nonzero leading coefficient)
static vec prem(vec a, const vec& b) {
    int db = (int)b.size() - 1;
    while ((int)a.size() - 1 >= db && a.size() > 0) {
        real f = a.back() / b.back();
        int shift = (int)a.size() - 1 - db;
        for (int i = 0; i <= db; ++i) a[shift + i] -= f * b[i];
        a.pop_back();
        if (a.empty()) break;
    }
    if (a.empty()) a.push_back(0.0L);
    ptrim(a);
    return a;
}

static int sign_changes(const std::vector<vec>& chain, real t) {
    int changes = 0;
    int prev = 0;
    for (const vec& p : chain) {
        real v = peval(p, t);
        int s = v > 0 ? 1 : (v < 0 ? -1 : 0);
        if (s == 0) continue;
        if (prev != 0 && s != prev) ++changes;
        prev = s;
    }
    return changes;
}

// Number of distinct real zeros of q in [0, 1] by Sturm's theorem, plus a
// direct check of the end points.
static int zeros_in_unit(vec q) {
    ptrim(q);
    if (q.size() <= 1) return fabsl(q[0]) > 0 ? 0 : 1;
    if (peval(q, 0.0L) == 0.0L || peval(q, 1.0L) == 0.0L) return 1;
    std::vector<vec> chain{q, pderiv(q)};
    while (chain.back().size() > 1 || fabsl(chain.back()[0]) > 0) {
        vec r = prem(chain[chain.size() - 2], chain.back());
        for (real& v : r) v = -v;
        real mx = 0.0L;
        for (real v : r) mx = std::max(mx, fabsl(v));
        if (mx == 0.0L) break;
        chain.push_back(r);
        if (r.size() == 1) break;
    }
    return sign_changes(chain, 0.0L) - sign_changes(chain, 1.0L);
}

// ------------------------------------------------------------- one Remez fit

struct Problem {
    int k;       // order approximated: F_k
    bool regionA;
    int kmax;    // weight rho_{A,kmax} in region A
    real a, b;   // interval
    real f(real x) const { return boys_ref(k, x); }
    real rho(real x) const { return regionA ? rho_A(kmax, x) : 1.0L; }
};

struct Fit {
    bool ok = false;
    int n = 0, m = 0;
    real E = 0;       // levelled error |E|
    real maxerr = 0;  // max |rho (f - r)| on the check grid
    vec p, q;         // in t = (x - a) / (b - a)... see scale below
};

// The fit variable is t = x / b (so that coefficients convert to x by pure
// scaling): the interval [a, b] maps to [a/b, 1].
struct Solver {
    const Problem& P;
    int n, m, N;
    real ta;  // a / b
    real wexp = 1.0L;  // the weight used is rho^wexp (continuation from 0 to 1)
    std::vector<real> grid;

    real rho(real x) const { return wexp == 1.0L ? P.rho(x) : powl(P.rho(x), wexp); }

    Solver(const Problem& pr, int n_, int m_) : P(pr), n(n_), m(m_), N(n_ + m_ + 2) {
        ta = P.a / P.b;
        const int K = 3000;
        for (int i = 0; i <= K; ++i) {  // Chebyshev-clustered grid in t
            real c = 0.5L * (1.0L - cosl(PI_L * i / K));
            grid.push_back(ta + (1.0L - ta) * c);
        }
    }

    real err(const vec& p, const vec& q, real t) const {
        real x = t * P.b;
        return rho(x) * (P.f(x) - peval(p, t) / peval(q, t));
    }

    // Step 2 + 3: solve at nodes t, return false if no pole-free solution.
    bool solve(const vec& t, vec& p, vec& q, real& E) const {
        vec f(N), rh(N), w(N);
        for (int i = 0; i < N; ++i) {
            real x = t[i] * P.b;
            f[i] = P.f(x);
            rh[i] = rho(x);
            real prod = 1.0L;
            for (int j = 0; j < N; ++j)
                if (j != i) prod *= (t[i] - t[j]);
            w[i] = 1.0L / prod;
        }
        const int sgn = (w[0] > 0) ? 1 : -1;  // w_i (-1)^i has the sign of w_0
        vec D(N);
        for (int i = 0; i < N; ++i) D[i] = fabsl(w[i]) / rh[i];
        // Orthonormal basis (values at nodes + monomial coefficients) by
        // Gram-Schmidt applied twice, in the inner product <g,h> = sum D g h.
        std::vector<vec> vals, coef;
        for (int kdeg = 0; kdeg <= m; ++kdeg) {
            vec v(N), c(m + 1, 0.0L);
            for (int i = 0; i < N; ++i) v[i] = powl(t[i], kdeg);
            c[kdeg] = 1.0L;
            for (int pass = 0; pass < 2; ++pass)
                for (size_t j = 0; j < vals.size(); ++j) {
                    real dot = 0.0L;
                    for (int i = 0; i < N; ++i) dot += D[i] * v[i] * vals[j][i];
                    for (int i = 0; i < N; ++i) v[i] -= dot * vals[j][i];
                    for (int l = 0; l <= m; ++l) c[l] -= dot * coef[j][l];
                }
            real nrm = 0.0L;
            for (int i = 0; i < N; ++i) nrm += D[i] * v[i] * v[i];
            nrm = sqrtl(nrm);
            if (!(nrm > 0)) return false;
            for (int i = 0; i < N; ++i) v[i] /= nrm;
            for (int l = 0; l <= m; ++l) c[l] /= nrm;
            vals.push_back(v);
            coef.push_back(c);
        }
        const int M = m + 1;
        vec A(M * M, 0.0L);
        for (int r = 0; r < M; ++r)
            for (int s = 0; s < M; ++s) {
                real acc = 0.0L;
                for (int i = 0; i < N; ++i) acc += w[i] * f[i] * vals[r][i] * vals[s][i];
                A[r * M + s] = acc;
            }
        vec d, V;
        jacobi(M, A, d, V);
        // candidate j: q = sum_r V[r][j] psi_r, E = sgn * d_j
        bool found = false;
        for (int j = 0; j < M && !found; ++j) {
            vec qc(m + 1, 0.0L);
            for (int r = 0; r < M; ++r)
                for (int l = 0; l <= m; ++l) qc[l] += V[r * M + j] * coef[r][l];
            // q on [ta, 1]: substitute t = ta + (1 - ta) u to test u in [0, 1]
            vec qu(m + 1, 0.0L);
            {
                // Horner-style composition q(ta + s u)
                vec acc{0.0L};
                for (int l = m; l >= 0; --l) {
                    vec nxt(acc.size() + 1, 0.0L);
                    for (size_t i = 0; i < acc.size(); ++i) {
                        nxt[i] += acc[i] * ta;
                        nxt[i + 1] += acc[i] * (1.0L - ta);
                    }
                    nxt[0] += qc[l];
                    acc = nxt;
                }
                acc.resize(m + 1);
                qu = acc;
            }
            if (zeros_in_unit(qu) != 0) continue;
            real Ej = sgn * d[j];
            // p through p(t_i) = q(t_i)(f_i - (-1)^i E / rho_i), least squares
            // in a basis orthonormal on the nodes (consistent system).
            vec rhs(N);
            for (int i = 0; i < N; ++i) rhs[i] = peval(qc, t[i]) * (f[i] - ((i & 1) ? -Ej : Ej) / rh[i]);
            std::vector<vec> pv, pc;
            vec pcoef(n + 1, 0.0L);
            for (int kdeg = 0; kdeg <= n; ++kdeg) {
                vec v(N), c(n + 1, 0.0L);
                for (int i = 0; i < N; ++i) v[i] = powl(t[i], kdeg);
                c[kdeg] = 1.0L;
                for (int pass = 0; pass < 2; ++pass)
                    for (size_t jj = 0; jj < pv.size(); ++jj) {
                        real dot = 0.0L;
                        for (int i = 0; i < N; ++i) dot += v[i] * pv[jj][i];
                        for (int i = 0; i < N; ++i) v[i] -= dot * pv[jj][i];
                        for (int l = 0; l <= n; ++l) c[l] -= dot * pc[jj][l];
                    }
                real nrm = 0.0L;
                for (int i = 0; i < N; ++i) nrm += v[i] * v[i];
                nrm = sqrtl(nrm);
                for (int i = 0; i < N; ++i) v[i] /= nrm;
                for (int l = 0; l <= n; ++l) c[l] /= nrm;
                real dot = 0.0L;
                for (int i = 0; i < N; ++i) dot += v[i] * rhs[i];
                for (int l = 0; l <= n; ++l) pcoef[l] += dot * c[l];
                pv.push_back(v);
                pc.push_back(c);
            }
            p = pcoef;
            q = qc;
            E = Ej;
            found = true;
        }
        return found;
    }

    real golden_max(const vec& p, const vec& q, real lo, real hi, int sgn) const {
        const real g = (sqrtl(5.0L) - 1.0L) / 2.0L;
        real c = hi - g * (hi - lo), d = lo + g * (hi - lo);
        real fc = sgn * err(p, q, c), fd = sgn * err(p, q, d);
        for (int it = 0; it < 60; ++it) {
            if (fc > fd) { hi = d; d = c; fd = fc; c = hi - g * (hi - lo); fc = sgn * err(p, q, c); }
            else { lo = c; c = d; fc = fd; d = lo + g * (hi - lo); fd = sgn * err(p, q, d); }
        }
        return 0.5L * (lo + hi);
    }

    // Remez iterations from the nodes t.  Returns 1 on convergence (fit in
    // out), 0 when the iteration breaks down (no pole-free solution, too few
    // alternating extrema), -1 when Step 6 proves the target unreachable.
    int iterate(vec& t, real target, Fit& out) const {
        vec p, q;
        real E = 0;
        for (int iter = 0; iter < 80; ++iter) {
            if (!solve(t, p, q, E)) return 0;  // Step 3 failed
            // Step 4: error on the grid
            std::vector<real> e(grid.size());
            real mx = 0.0L;
            for (size_t i = 0; i < grid.size(); ++i) {
                e[i] = err(p, q, grid[i]);
                mx = std::max(mx, fabsl(e[i]));
            }
            if (mx - fabsl(E) <= 2e-4L * fabsl(E)) {
                out.ok = true;
                out.E = fabsl(E);
                out.maxerr = mx;
                out.p = p;
                out.q = q;
                return 1;
            }
            // Step 5: local extrema of e on the grid (end points included),
            // refined by golden section, grouped by sign.
            std::vector<real> ext;
            for (size_t i = 0; i < grid.size(); ++i) {
                bool left = (i == 0) || fabsl(e[i]) >= fabsl(e[i - 1]);
                bool right = (i + 1 == grid.size()) || fabsl(e[i]) >= fabsl(e[i + 1]);
                if (!(left && right) || e[i] == 0) continue;
                real x = grid[i];
                if (i > 0 && i + 1 < grid.size())
                    x = golden_max(p, q, grid[i - 1], grid[i + 1], e[i] > 0 ? 1 : -1);
                ext.push_back(x);
            }
            // alternating subsequence: within runs of equal sign keep the largest
            std::vector<real> alt;
            std::vector<real> av;
            for (real x : ext) {
                real v = err(p, q, x);
                if (!alt.empty() && ((v > 0) == (av.back() > 0))) {
                    if (fabsl(v) > fabsl(av.back())) { alt.back() = x; av.back() = v; }
                } else {
                    alt.push_back(x);
                    av.push_back(v);
                }
            }
            if ((int)alt.size() < N) return 0;
            // trim to N keeping the global maximum: drop the smaller end
            while ((int)alt.size() > N) {
                if (fabsl(av.front()) < fabsl(av.back())) { alt.erase(alt.begin()); av.erase(av.begin()); }
                else { alt.pop_back(); av.pop_back(); }
            }
            // Step 6: de la Vallee-Poussin bound (only meaningful with the full weight)
            real mn = 1e300L;
            for (real v : av) mn = std::min(mn, fabsl(v));
            if (wexp == 1.0L && mn > target) { out.ok = false; out.E = mn; return -1; }
            t = alt;
        }
        return 0;
    }

    void initial_nodes(vec& t, int attempt, unsigned long long& rng) const {
        auto urand = [&rng]() {
            rng ^= rng << 13;
            rng ^= rng >> 7;
            rng ^= rng << 17;
            return (real)(rng >> 11) * (1.0L / 9007199254740992.0L);
        };
        for (int i = 0; i < N; ++i) {
            real c = 0.5L * (1.0L - cosl(PI_L * i / (N - 1)));
            if (attempt > 0 && i > 0 && i < N - 1) c += (urand() - 0.5L) * 0.4L / N;
            t[i] = ta + (1.0L - ta) * c;
        }
        std::sort(t.begin(), t.end());
    }

    Fit run(real target, unsigned seed) {
        Fit out;
        out.n = n;
        out.m = m;
        vec t(N);
        unsigned long long rng = 0x9E3779B97F4A7C15ULL ^ seed;  // local xorshift: deterministic restarts
        // Step 1 with restarts (perturbed Chebyshev nodes)
        for (int attempt = 0; attempt < 6; ++attempt) {
            initial_nodes(t, attempt, rng);
            wexp = 1.0L;
            const int r = iterate(t, target, out);
            if (r != 0) return out;
        }
        // Continuation in the weight for strongly weighted problems: solve
        // with rho^s, s = 0, 1/4, ..., 1, each stage starting from the
        // previous stage's equioscillation nodes.
        initial_nodes(t, 0, rng);
        for (int stage = 0; stage <= 4; ++stage) {
            wexp = stage / 4.0L;
            Fit tmp;
            tmp.n = n;
            tmp.m = m;
            const int r = iterate(t, target, tmp);
            if (r != 1) {
                wexp = 1.0L;
                out.ok = false;
                if (r == -1) out.E = tmp.E;
                return out;
            }
            if (stage == 4) { wexp = 1.0L; return tmp; }
            // the converged nodes of this stage: alternating maxima of its error
            vec nodes;
            std::vector<real> vals;
            for (size_t i = 0; i < grid.size(); ++i) {
                const real v = err(tmp.p, tmp.q, grid[i]);
                bool left = (i == 0) || fabsl(v) >= fabsl(err(tmp.p, tmp.q, grid[i - 1]));
                bool right = (i + 1 == grid.size()) || fabsl(v) >= fabsl(err(tmp.p, tmp.q, grid[i + 1]));
                if (!(left && right) || v == 0) continue;
                if (!nodes.empty() && ((v > 0) == (vals.back() > 0))) {
                    if (fabsl(v) > fabsl(vals.back())) { nodes.back() = grid[i]; vals.back() = v; }
                } else {
                    nodes.push_back(grid[i]);
                    vals.push_back(v);
                }
            }
            while ((int)nodes.size() > N) {
                if (fabsl(vals.front()) < fabsl(vals.back())) { nodes.erase(nodes.begin()); vals.erase(vals.begin()); }
                else { nodes.pop_back(); vals.pop_back(); }
            }
            if ((int)nodes.size() < N) { wexp = 1.0L; return out; }
            t = nodes;
        }
        wexp = 1.0L;
        return out;
    }
};

// ------------------------------------------------------------- Walsh-table search

static Fit walsh_search(const Problem& P, real target, int dmax) {
    for (int d = 0; d <= dmax; ++d) {
        Fit best;
        for (int n = d; n >= 0; --n) {
            int m = d - n;
            Solver S(P, n, m);
            Fit f = S.run(target, 1234u + 17u * n + 31u * m);
            if (f.ok && f.maxerr <= target && (!best.ok || f.maxerr < best.maxerr)) best = f;
        }
        if (best.ok) return best;
    }
    return Fit{};
}

// ------------------------------------------------------------- FP32 evaluation check

struct Tier {
    int kmax;
    float x0, x1;
    std::vector<float> ap, aq, bp, bq;  // coefficients in x, lowest degree first
    vec eap, eaq, ebp, ebq;             // the same before rounding (monic in x)
};

// coefficient of t^i with t = x / b  ->  coefficient of x^i = c_i / b^i
static vec to_x(const vec& c, real b) {
    vec out;
    for (size_t i = 0; i < c.size(); ++i) out.push_back(c[i] / powl(b, (real)i));
    return out;
}

// scale p and q (already in x) so that q is monic in x, then round to FP32
static void monic_float(vec p, vec q, std::vector<float>* pf, std::vector<float>* qf, vec* pe, vec* qe) {
    real lead = q.back();
    pf->clear();
    qf->clear();
    pe->clear();
    qe->clear();
    for (real v : p) { pf->push_back((float)(v / lead)); pe->push_back(v / lead); }
    for (size_t i = 0; i + 1 < q.size(); ++i) { qf->push_back((float)(q[i] / lead)); qe->push_back(q[i] / lead); }
    qf->push_back(1.0f);
    qe->push_back(1.0L);
}

static float horner_f(const std::vector<float>& c, float x) {
    float v = c.back();
    for (int i = (int)c.size() - 2; i >= 0; --i) v = fmaf(v, x, c[i]);
    return v;
}

// The kernel's e^{-x}: Cody and Waite's reduction x = n ln2 + r and the
// degree-7 Taylor polynomial of e^{-r}, in the same float operations.
static float exp_neg_f(float x) {
    const float t = fmaf(x, 1.4426950216293335f, 12582912.0f);
    const float n = t - 12582912.0f;
    float r = fmaf(-n, 0.693115234375f, x);
    r = fmaf(-n, 3.194618329871446e-05f, r);
    float p = -1.98412701e-04f;
    for (float c : {1.38888892e-03f, -8.33333377e-03f, 4.16666679e-02f, -1.66666672e-01f, 0.5f, -1.0f, 1.0f})
        p = fmaf(p, r, c);
    return ldexpf(p, -(int)n);
}

// Algorithm 1 in FP32 with the kernel's operation order; F[0..kmax].  The
// kernel's quotient, reciprocal and inverse square root (hardware seed plus
// one correction, within about an ulp) are modelled by the correctly rounded
// operations.
static void eval_f32(const Tier& T, float x, float* F) {
    const int K = T.kmax;
    const bool inA = x < T.x0, inC = x >= T.x1;
    const float r = 1.0f / sqrtf(x);
    float y0;
    if (inC) y0 = 0.88622692545275801365f * r;
    else if (inA) y0 = horner_f(T.ap, x) / horner_f(T.aq, x);
    else y0 = horner_f(T.bp, x) / horner_f(T.bq, x);
    const float e = inC ? 0.0f : exp_neg_f(x);
    const float two_x = x + x, inv2x = 1.0f / two_x;
    float y[40];
    y[0] = y0;
    for (int j = 0; j < K; ++j) {
        const int l = K - 1 - j;
        const float a = inA ? two_x : (float)(2 * j + 1);
        const float c = inA ? 1.0f / (float)(2 * l + 1) : inv2x;
        const float s = inA ? e : -e;
        y[j + 1] = fmaf(a, y[j], s) * c;
    }
    for (int k = 0; k <= K; ++k) F[k] = inA ? y[K - k] : y[k];
}

static real verify(const Tier& T, std::vector<real>* per_k) {
    const int K = T.kmax;
    per_k->assign(K + 1, 0.0L);
    real worst = 0.0L;
    std::vector<float> xs;
    for (int i = 0; i <= 20000; ++i) xs.push_back((float)(1.1L * T.x1 * i / 20000.0L));
    for (int i = 0; i <= 4000; ++i) xs.push_back((float)expl(logl(1e-8L) + (logl(1e4L) - logl(1e-8L)) * i / 4000.0L));
    for (float b : {T.x0, T.x1}) {
        float v = b;
        for (int s = 0; s < 8; ++s) v = nextafterf(v, 0.0f);
        for (int s = 0; s < 17; ++s) { xs.push_back(v); v = nextafterf(v, 1e30f); }
    }
    float F[40];
    for (float x : xs) {
        eval_f32(T, x, F);
        for (int k = 0; k <= K; ++k) {
            real e = fabsl((real)F[k] - boys_ref(k, (real)x));
            (*per_k)[k] = std::max((*per_k)[k], e);
            worst = std::max(worst, e);
        }
    }
    return worst;
}

// ------------------------------------------------------------- driver

static void emit_vec(FILE* o, const std::vector<float>& v, int len) {
    fprintf(o, "{ ");
    for (int i = 0; i < len; ++i) fprintf(o, "%s%.9ef", i ? ", " : "", i < (int)v.size() ? (double)v[i] : 0.0);
    fprintf(o, " }");
}

// ------------------------------------------------------------- FP64 tables (report)
//
// `boys_remez --fp64 KFIRST KLAST [--with-b]` regenerates the paper's FP64 table
// set for eps_tol = 5e-14 (Appendix D): x0 by Eq. x0 for kmax = 32, x1 by Eq. x1,
// r_{A,k} on [0, x0) with weight rho_{A,k} for k in [KFIRST, KLAST], and (with
// --with-b) r_B on [x0, x1).  For each fit it prints the chosen (n, m) and the
// levelled error, and checks Algorithm 1 evaluated in double precision with the
// fitted anchor (rounded to double): the downward recurrence from r_{A,k} over
// [0, x0) for every order 0..k, or the upward one from r_B over [x0, x1) for
// orders 0..32.  The product's FP64 tables stay the printed ones; this is a
// check of the generator against the paper's published result.

static double horner_d(const std::vector<double>& c, double x) {
    double v = c.back();
    for (int i = (int)c.size() - 2; i >= 0; --i) v = fma(v, x, c[i]);
    return v;
}

static real check_A_fp64(int k, const std::vector<double>& p, const std::vector<double>& q, double x0) {
    real worst = 0.0L;
    for (int i = 0; i < 6000; ++i) {
        const double x = x0 * (i + 0.5) / 6000.0;
        double F = horner_d(p, x) / horner_d(q, x);
        const double e = exp(-x);
        worst = std::max(worst, fabsl((real)F - boys_ref(k, x)));
        for (int l = k - 1; l >= 0; --l) {
            F = fma(2.0 * x, F, e) / (double)(2 * l + 1);
            worst = std::max(worst, fabsl((real)F - boys_ref(l, x)));
        }
    }
    return worst;
}

static real check_B_fp64(const std::vector<double>& p, const std::vector<double>& q, double x0, double x1) {
    real worst = 0.0L;
    for (int i = 0; i < 6000; ++i) {
        const double x = x0 + (x1 - x0) * (i + 0.5) / 6000.0;
        double F = horner_d(p, x) / horner_d(q, x);
        const double e = exp(-x);
        worst = std::max(worst, fabsl((real)F - boys_ref(0, x)));
        for (int l = 0; l < 32; ++l) {
            F = ((double)(2 * l + 1) * F - e) / (2.0 * x);
            worst = std::max(worst, fabsl((real)F - boys_ref(l + 1, x)));
        }
    }
    return worst;
}

static int run_fp64(int kfirst, int klast, bool with_b) {
    const real eps = 5e-14L;
    const real x0 = x0_of(32), x1 = x1_of(32, eps);
    printf("x0 %.17Lg\nx1 %.17Lg\n", x0, x1);
    const int nfit = klast - kfirst + 1 + (with_b ? 1 : 0);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int t = 0; t < nfit; ++t) {
        const bool isB = with_b && t == nfit - 1;
        Problem P = isB ? Problem{0, false, 32, x0, x1} : Problem{kfirst + t, true, kfirst + t, 0.0L, x0};
        const Fit f = walsh_search(P, eps, 22);
        if (!f.ok) {
#pragma omp critical
            {
                printf("%s %d FAILED\n", isB ? "B" : "A", isB ? 0 : kfirst + t);
                fflush(stdout);
            }
            ++bad;
            continue;
        }
        const real b = isB ? x1 : x0;
        vec px = to_x(f.p, b), qx = to_x(f.q, b);
        const real lead = qx.back();
        std::vector<double> pd, qd;
        for (real v : px) pd.push_back((double)(v / lead));
        for (real v : qx) qd.push_back((double)(v / lead));
        const real err = isB ? check_B_fp64(pd, qd, (double)x0, (double)x1)
                             : check_A_fp64(kfirst + t, pd, qd, (double)x0);
#pragma omp critical
        {
            printf("%s %d n %d m %d E %.4Le fp64_alg1_max_err %.4Le\n", isB ? "B" : "A", isB ? 0 : kfirst + t,
                   f.n, f.m, f.E, err);
            fflush(stdout);
        }
    }
    return bad ? 1 : 0;
}

int main(int argc, char** argv) {
    if (argc > 1 && strcmp(argv[1], "--fp64") == 0) {
        const int kf = argc > 2 ? atoi(argv[2]) : 0, kl = argc > 3 ? atoi(argv[3]) : 32;
        const bool wb = argc > 4 && strcmp(argv[4], "--with-b") == 0;
        return run_fp64(kf, kl, wb);
    }
    const real eps_total = 1e-6L;   // FP32-tier tolerance (absolute)
    real eps_fit = 3e-7L;           // minimax target for the rational anchors
    const real eps_c = 3e-7L;       // region-C asymptotic budget (Eq. x1)
    const real budget = 0.9L * eps_total;
    int kfirst = 0, klast = 32;
    if (argc > 2) { kfirst = atoi(argv[1]); klast = atoi(argv[2]); }
    std::vector<Tier> tiers(klast + 1);
    std::vector<std::vector<real>> reports(klast + 1);
    std::vector<real> fitE(2 * (klast + 1));
#pragma omp parallel for schedule(dynamic, 1)
    for (int kmax = kfirst; kmax <= klast; ++kmax) {
        real target = eps_fit;
        for (int attempt = 0; attempt < 6; ++attempt) {
            Tier T;
            T.kmax = kmax;
            real x0 = x0_of(kmax), x1 = x1_of(kmax, eps_c);
            T.x0 = (float)x0;
            T.x1 = (float)x1;
            Problem PA{kmax, true, kmax, 0.0L, (real)T.x0};
            Problem PB{0, false, kmax, (real)T.x0, (real)T.x1};
            Fit fa = walsh_search(PA, target, 24);
            Fit fb = walsh_search(PB, target, 24);
            if (!fa.ok || !fb.ok) { target *= 0.5L; continue; }
            monic_float(to_x(fa.p, PA.b), to_x(fa.q, PA.b), &T.ap, &T.aq, &T.eap, &T.eaq);
            monic_float(to_x(fb.p, PB.b), to_x(fb.q, PB.b), &T.bp, &T.bq, &T.ebp, &T.ebq);
            std::vector<real> per_k;
            real worst = verify(T, &per_k);
            fprintf(stderr, "kmax=%2d x0=%.6f x1=%.6f A(%d,%d) E=%.3Le  B(%d,%d) E=%.3Le  fp32 worst=%.3Le (target %.2Le)\n",
                    kmax, (double)T.x0, (double)T.x1, fa.n, fa.m, fa.E, fb.n, fb.m, fb.E, worst, target);
            if (worst <= budget) {
                tiers[kmax] = T;
                reports[kmax] = per_k;
                fitE[2 * kmax] = fa.E;
                fitE[2 * kmax + 1] = fb.E;
                break;
            }
            target *= 0.5L;
        }
        if (tiers[kmax].ap.empty()) fprintf(stderr, "kmax=%d: FAILED to meet the budget\n", kmax);
    }
    for (int kmax = kfirst; kmax <= klast; ++kmax)
        if (tiers[kmax].ap.empty()) return 1;

    size_t pl = 0, ql = 0, bpl = 0, bql = 0;
    for (int kmax = kfirst; kmax <= klast; ++kmax) {
        pl = std::max(pl, tiers[kmax].ap.size());
        ql = std::max(ql, tiers[kmax].aq.size());
        bpl = std::max(bpl, tiers[kmax].bp.size());
        bql = std::max(bql, tiers[kmax].bq.size());
    }
    FILE* o = stdout;
    fprintf(o, "// FP32-tier tables for the Boys functions (absolute tolerance 1e-6), one set per kmax.\n");
    fprintf(o, "// Generated by csrc/remez/boys_remez.cpp (rational Remez in extended precision,\n");
    fprintf(o, "// Walsh-table degree choice); do not edit.  Index i multiplies x^i; denominators\n");
    fprintf(o, "// are monic.  x0 by Eq. x0, x1 by Eq. x1 with a 3e-7 region-C budget.\n");
    fprintf(o, "#pragma once\n\n#define BOYS_F32_KMAX %d\n", klast);
    fprintf(o, "#define BOYS_F32_AP_LEN %zu\n#define BOYS_F32_AQ_LEN %zu\n#define BOYS_F32_BP_LEN %zu\n#define BOYS_F32_BQ_LEN %zu\n",
            pl, ql, bpl, bql);
    fprintf(o, "#define BOYS_F32_X0_INIT { ");
    for (int k = kfirst; k <= klast; ++k) fprintf(o, "%s%.9ef", k ? ", " : "", (double)tiers[k].x0);
    fprintf(o, " }\n#define BOYS_F32_X1_INIT { ");
    for (int k = kfirst; k <= klast; ++k) fprintf(o, "%s%.9ef", k ? ", " : "", (double)tiers[k].x1);
    fprintf(o, " }\n#define BOYS_F32_AN_INIT { ");
    for (int k = kfirst; k <= klast; ++k) fprintf(o, "%s%zu", k ? ", " : "", tiers[k].ap.size() - 1);
    fprintf(o, " }\n#define BOYS_F32_AM_INIT { ");
    for (int k = kfirst; k <= klast; ++k) fprintf(o, "%s%zu", k ? ", " : "", tiers[k].aq.size() - 1);
    fprintf(o, " }\n#define BOYS_F32_BN_INIT { ");
    for (int k = kfirst; k <= klast; ++k) fprintf(o, "%s%zu", k ? ", " : "", tiers[k].bp.size() - 1);
    fprintf(o, " }\n#define BOYS_F32_BM_INIT { ");
    for (int k = kfirst; k <= klast; ++k) fprintf(o, "%s%zu", k ? ", " : "", tiers[k].bq.size() - 1);
    fprintf(o, " }\n");
    const char* names[4] = {"AP", "AQ", "BP", "BQ"};
    for (int t = 0; t < 4; ++t) {
        fprintf(o, "#define BOYS_F32_%s_INIT { \\\n", names[t]);
        for (int k = kfirst; k <= klast; ++k) {
            const std::vector<float>& v = t == 0 ? tiers[k].ap : t == 1 ? tiers[k].aq : t == 2 ? tiers[k].bp : tiers[k].bq;
            size_t len = t == 0 ? pl : t == 1 ? ql : t == 2 ? bpl : bql;
            fprintf(o, "  ");
            emit_vec(o, v, (int)len);
            fprintf(o, ", \\\n");
        }
        fprintf(o, "}\n");
    }
    // The unrounded minimax coefficients (21 significant digits), for tests of
    // the equioscillation property; the kernel uses only the FP32 tables.
    const char* enames[4] = {"AP", "AQ", "BP", "BQ"};
    for (int t = 0; t < 4; ++t) {
        fprintf(o, "#define BOYS_F32_%s_EXT { \\\n", enames[t]);
        for (int k = kfirst; k <= klast; ++k) {
            const vec& v = t == 0 ? tiers[k].eap : t == 1 ? tiers[k].eaq : t == 2 ? tiers[k].ebp : tiers[k].ebq;
            fprintf(o, "  { ");
            for (size_t i = 0; i < v.size(); ++i) fprintf(o, "%s%.21Le", i ? ", " : "", v[i]);
            fprintf(o, " }, \\\n");
        }
        fprintf(o, "}\n");
    }
    fprintf(o, "// Verified in host FP32 arithmetic against extended-precision references\n");
    fprintf(o, "// (max abs error over all orders, dense grid on [0, 1.1 x1], log grid to 1e4,\n");
    fprintf(o, "// 17 floats around each boundary), and levelled minimax errors |E| of the fits:\n");
    for (int k = kfirst; k <= klast; ++k) {
        real w = 0;
        for (real v : reports[k]) w = std::max(w, v);
        fprintf(o, "//   kmax=%2d  worst %.3Le   |E_A| %.3Le  |E_B| %.3Le\n", k, w, fitE[2 * k], fitE[2 * k + 1]);
    }
    return 0;
}
