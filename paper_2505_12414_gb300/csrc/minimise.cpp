// minimise.cpp -- host variable-metric minimiser for the unbinned NLL.
//
// The paper minimises with Minuit2's Migrad on the host, feeding it the analytic gradient
// computed on the accelerator, and takes uncertainties from the inverse Hessian (HESSE)
// (paper Sec. 2.1 and Sec. 3.1).  This is the project's own minimiser of that kind,
// written from the textbook descriptions:
//   * BFGS update of the inverse Hessian (Broyden, Fletcher, Goldfarb, Shanno 1970), with
//     the initial matrix either diag(step^2) or the inverse of a finite-difference Hessian
//     of the analytic gradient (the "strategy" of Minuit);
//   * line search for the Armijo sufficient-decrease condition with safeguarded quadratic
//     backtracking, extrapolating while the curvature condition is not met;
//   * bounded parameters through the sine transform described in the Minuit manual:
//     external = lo + (hi - lo) (sin(internal) + 1) / 2;
//   * convergence on the estimated distance to minimum EDM = g^T V g / 2;
//   * optionally a finite-difference Hessian of the analytic gradient at the minimum,
//     Newton polish steps with it, and the covariance as its inverse;
//   * or, where the objective supplies them, the analytic Hessian (for the start matrix,
//     the polish and the covariance) and the weighted-fit sandwich covariance
//     H^-1 W H^-1, W = sum w^2 s s^T (paper Sec. 2.1 asks for both);
//   * or (strategy 4) damped Newton steps with the analytic Hessian at every iterate, which
//     takes far fewer passes over the events where a pass with second derivatives costs about
//     what one without does (small samples, where each pass is launch latency).
#include "minimise.h"
#include "trace.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace gbnll {

bool spd_inverse(int n, const double* a, double* inv)
{
    // Cholesky a = L L^T, then inv = L^-T L^-1
    std::vector<double> L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0) || !isfinite(d)) return false;
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = a[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    // Linv (lower triangular)
    std::vector<double> Li((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        Li[i * n + i] = 1.0 / L[i * n + i];
        for (int j = 0; j < i; ++j) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s -= L[i * n + k] * Li[k * n + j];
            Li[i * n + j] = s / L[i * n + i];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int k = i; k < n; ++k) s += Li[k * n + i] * Li[k * n + j];
            inv[i * n + j] = inv[j * n + i] = s;
        }
    return true;
}

namespace {

struct Problem {
    const Objective& fn;
    int n;        // external parameters
    int nf;       // free parameters
    std::vector<int> idx;   // free -> external index
    std::vector<double> lo, hi, base;  // bounds, full external vector (fixed values)
    std::vector<char> bounded;
    int n_eval = 0;

    Problem(const Objective& f, int n_) : fn(f), n(n_) {}

    double to_ext(int i, double x) const
    {
        int k = idx[i];
        if (!bounded[k]) return x;
        return lo[k] + (hi[k] - lo[k]) * 0.5 * (sin(x) + 1.0);
    }
    double jac(int i, double x) const
    {
        int k = idx[i];
        return bounded[k] ? (hi[k] - lo[k]) * 0.5 * cos(x) : 1.0;
    }
    double to_int(int i, double e) const
    {
        int k = idx[i];
        if (!bounded[k]) return e;
        double u = 2.0 * (e - lo[k]) / (hi[k] - lo[k]) - 1.0;
        u = std::min(std::max(u, -1.0 + 1e-10), 1.0 - 1e-10);  // keep the transform invertible
        return asin(u);
    }
    void external(const std::vector<double>& x, std::vector<double>& th) const
    {
        th = base;
        for (int i = 0; i < nf; ++i) th[idx[i]] = to_ext(i, x[i]);
    }
    // internal objective; returns nll_status
    int eval_int(const std::vector<double>& x, double& f, std::vector<double>& g)
    {
        std::vector<double> th, ge(n);
        external(x, th);
        ++n_eval;
        int st = fn(th.data(), &f, ge.data());
        if (st != NLL_OK) return st;
        if (!isfinite(f)) return NLL_ERR_NONPOSITIVE_PDF;
        g.resize(nf);
        for (int i = 0; i < nf; ++i) {
            g[i] = ge[idx[i]] * jac(i, x[i]);
            if (!isfinite(g[i])) return NLL_ERR_NONPOSITIVE_PDF;
        }
        return NLL_OK;
    }
    int eval_ext(const std::vector<double>& th_free, double& f, std::vector<double>& g)
    {
        std::vector<double> th = base, ge(n);
        for (int i = 0; i < nf; ++i) th[idx[i]] = th_free[i];
        ++n_eval;
        int st = fn(th.data(), &f, ge.data());
        if (st != NLL_OK) return st;
        if (!isfinite(f)) return NLL_ERR_NONPOSITIVE_PDF;
        g.resize(nf);
        for (int i = 0; i < nf; ++i) g[i] = ge[idx[i]];
        return NLL_OK;
    }
};

double dot(const std::vector<double>& a, const std::vector<double>& b)
{
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

void matvec(int n, const std::vector<double>& M, const std::vector<double>& v, std::vector<double>& out)
{
    out.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += M[i * n + j] * v[j];
        out[i] = s;
    }
}

// finite-difference Hessian of the gradient; eval(k, +/-h) supplies the gradient
template <class G>
bool fd_hessian(int n, const std::vector<double>& h, G grad_at, std::vector<double>& H)
{
    H.assign((size_t)n * n, 0.0);
    std::vector<double> gp, gm;
    for (int k = 0; k < n; ++k) {
        if (!grad_at(k, +h[k], gp) || !grad_at(k, -h[k], gm)) return false;
        for (int j = 0; j < n; ++j) H[j * n + k] = (gp[j] - gm[j]) / (2.0 * h[k]);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            double s = 0.5 * (H[i * n + j] + H[j * n + i]);
            H[i * n + j] = H[j * n + i] = s;
        }
    return true;
}

// Damped Newton minimisation with the analytic Hessian at every iterate (strategy 4).  Each
// evaluation is one pass that returns f, g and H together; in internal coordinates the
// Hessian is J H J + diag(dF/dext d2ext/dx2) (sine transform), and the step -H_int^-1 g_int is
// taken with the Armijo backtracking of the quasi-Newton line search.  Where H_int is not
// positive definite the step falls back to the scaled gradient -diag(s^2) g.  At convergence
// (EDM with the exact Hessian below tol_edm) the covariance is the inverse external Hessian
// of the final point, or the sandwich H^-1 W H^-1 with hessian 3: no further pass is needed.
// For samples whose evaluations cost about the same with or without second derivatives (small,
// latency-bound samples) this takes a few passes where the quasi-Newton route takes many.
struct NewtonPoint {
    std::vector<double> x, th_free, g_ext, H_ext, W_ext;
    double f = 0.0;
};

int newton_minimise(Problem& P, const HessianFn& hess, const fit_options& opt, std::vector<double> x,
                    const std::vector<double>& sint, const double* theta0, fit_result* out)
{
    const int n = P.n, nf = P.nf;
    const bool sandwich = opt.hessian == 3;
    std::vector<double> th, gn(n), Hn((size_t)n * n), Wn(sandwich ? (size_t)n * n : 0);  // reused every pass
    auto eval_at = [&](const std::vector<double>& xi, NewtonPoint& pt) -> int {
        P.external(xi, th);
        ++P.n_eval;
        double f;
        int st = hess(th.data(), &f, gn.data(), Hn.data(), sandwich ? Wn.data() : nullptr);
        if (st != NLL_OK) return st;
        if (!isfinite(f)) return NLL_ERR_NONPOSITIVE_PDF;
        pt.x = xi;
        pt.f = f;
        pt.th_free.resize(nf);
        pt.g_ext.resize(nf);
        pt.H_ext.resize((size_t)nf * nf);
        if (sandwich) pt.W_ext.resize((size_t)nf * nf);
        for (int i = 0; i < nf; ++i) {
            pt.th_free[i] = th[P.idx[i]];
            pt.g_ext[i] = gn[P.idx[i]];
            if (!isfinite(pt.g_ext[i])) return NLL_ERR_NONPOSITIVE_PDF;
            for (int j = 0; j < nf; ++j) {
                pt.H_ext[i * nf + j] = Hn[(size_t)P.idx[i] * n + P.idx[j]];
                if (sandwich) pt.W_ext[i * nf + j] = Wn[(size_t)P.idx[i] * n + P.idx[j]];
            }
        }
        return NLL_OK;
    };
    NewtonPoint cur;
    int st = eval_at(x, cur);
    if (st != NLL_OK) {
        out->status = st;
        out->n_eval = P.n_eval;
        return st;
    }
    std::vector<double> gi(nf), Hi((size_t)nf * nf), Vi((size_t)nf * nf), p(nf), Vg;
    double edm = INFINITY;
    bool converged = false, have_inverse = false;
    int iter = 0;
    for (;;) {
        // internal gradient and Hessian at the current point
        for (int i = 0; i < nf; ++i) {
            const double Ji = P.jac(i, cur.x[i]);
            gi[i] = cur.g_ext[i] * Ji;
            for (int j = 0; j < nf; ++j) Hi[i * nf + j] = Ji * cur.H_ext[i * nf + j] * P.jac(j, cur.x[j]);
            const int k = P.idx[i];
            if (P.bounded[k]) Hi[i * nf + i] += cur.g_ext[i] * (-(P.hi[k] - P.lo[k]) * 0.5 * sin(cur.x[i]));
        }
        have_inverse = spd_inverse(nf, Hi.data(), Vi.data());
        if (have_inverse) {
            matvec(nf, Vi, gi, Vg);
            edm = 0.5 * dot(gi, Vg);
            for (int i = 0; i < nf; ++i) p[i] = -Vg[i];
        } else {
            edm = INFINITY;
            for (int i = 0; i < nf; ++i) p[i] = -sint[i] * sint[i] * gi[i];
        }
        converged = have_inverse && edm < opt.tol_edm;
        if (converged || iter >= opt.max_iter) break;
        ++iter;
        const double gp = dot(gi, p);
        if (!(gp < 0.0)) break;
        // Armijo backtracking (every trial is a full pass: its Hessian serves the next step)
        const double c1 = 1e-4;
        double alpha = 1.0;
        bool ok = false;
        NewtonPoint trial;
        std::vector<double> xn(nf);
        for (int ls = 0; ls < 40; ++ls) {
            for (int i = 0; i < nf; ++i) xn[i] = cur.x[i] + alpha * p[i];
            const int s2 = eval_at(xn, trial);
            if (s2 == NLL_OK && trial.f <= cur.f + c1 * alpha * gp) {
                ok = true;
                break;
            }
            double anew;
            if (s2 == NLL_OK && isfinite(trial.f)) {
                const double denom = 2.0 * (trial.f - cur.f - gp * alpha);
                anew = denom > 0.0 ? -gp * alpha * alpha / denom : 0.5 * alpha;
                anew = std::min(std::max(anew, 0.1 * alpha), 0.5 * alpha);
            } else {
                anew = 0.25 * alpha;
            }
            alpha = anew;
        }
        if (!ok) break;
        const double fprev = cur.f;
        cur = trial;
        // an accepted step that no longer lowers the NLL (its change is below the rounding of
        // the sum): the exact EDM of this point decides convergence below
        if (!(cur.f < fprev) && iter > 2) break;
    }
    // external covariance at the final point: H^-1, or H^-1 W H^-1 (hessian 3)
    std::vector<double> C((size_t)nf * nf, 0.0), He_inv((size_t)nf * nf);
    if (spd_inverse(nf, cur.H_ext.data(), He_inv.data())) {
        if (sandwich) {
            std::vector<double> T((size_t)nf * nf, 0.0);
            for (int i = 0; i < nf; ++i)
                for (int k = 0; k < nf; ++k)
                    for (int j = 0; j < nf; ++j) T[i * nf + j] += He_inv[i * nf + k] * cur.W_ext[k * nf + j];
            for (int i = 0; i < nf; ++i)
                for (int j = 0; j < nf; ++j) {
                    double sacc = 0.0;
                    for (int k = 0; k < nf; ++k) sacc += T[i * nf + k] * He_inv[k * nf + j];
                    C[i * nf + j] = sacc;
                }
        } else {
            C = He_inv;
        }
        std::vector<double> d;
        matvec(nf, He_inv, cur.g_ext, d);
        edm = 0.5 * dot(cur.g_ext, d);
        converged = edm < opt.tol_edm;
    } else {
        converged = false;
    }
    for (int k = 0; k < n; ++k) out->theta[k] = theta0[k];
    for (int i = 0; i < nf; ++i) out->theta[P.idx[i]] = cur.th_free[i];
    for (int i = 0; i < nf; ++i) {
        for (int j = 0; j < nf; ++j) out->cov[P.idx[i] * n + P.idx[j]] = C[i * nf + j];
        out->err[P.idx[i]] = sqrt(std::max(C[i * nf + i], 0.0));
    }
    out->nll = cur.f;
    out->edm = edm;
    out->n_eval = P.n_eval;
    out->n_iter = iter;
    out->status = converged ? NLL_OK : NLL_ERR_NOT_CONVERGED;
    return out->status;
}

}  // namespace

int bfgs_minimise(const Objective& fn, int n, const double* theta0, const double* lo, const double* hi,
                  const double* step, const int* fixed, const fit_options* opt_in, fit_result* out,
                  const HessianFn* hess)
{
    GBNLL_TRACE("minimiser");
    fit_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        memset(&opt, 0, sizeof opt);
    if (!(opt.tol_edm > 0.0)) opt.tol_edm = 1e-8;
    if (opt.max_iter <= 0) opt.max_iter = 500;
    memset(out, 0, sizeof(*out));
    if (n <= 0 || n > FIT_MAXPAR || !theta0 || opt.strategy < 0 || opt.strategy > 4 || opt.strategy == 3 ||
        opt.hessian < 0 || opt.hessian > 3 || ((opt.strategy >= 2 || opt.hessian >= 2) && !hess)) {
        out->status = NLL_ERR_ARG;
        return NLL_ERR_ARG;
    }
    for (int k = 0; k < n; ++k) out->theta[k] = theta0[k];

    Problem P(fn, n);
    P.lo.assign(n, 0.0);
    P.hi.assign(n, 0.0);
    P.bounded.assign(n, 0);
    P.base.assign(theta0, theta0 + n);
    std::vector<double> s0;
    for (int k = 0; k < n; ++k) {
        if (!isfinite(theta0[k])) {
            out->status = NLL_ERR_ARG;
            return NLL_ERR_ARG;
        }
        if (lo && hi && lo[k] < hi[k] && isfinite(lo[k]) && isfinite(hi[k])) {
            P.bounded[k] = 1;
            P.lo[k] = lo[k];
            P.hi[k] = hi[k];
        }
        if (fixed && fixed[k]) continue;
        P.idx.push_back(k);
        double st = step && step[k] > 0.0 ? step[k] : std::max(1e-3 * fabs(theta0[k]), 1e-3);
        s0.push_back(st);
    }
    P.nf = (int)P.idx.size();
    const int nf = P.nf;
    if (nf == 0) {
        std::vector<double> g;
        double f;
        std::vector<double> empty;
        int st = P.eval_ext(empty, f, g);
        out->nll = f;
        out->n_eval = P.n_eval;
        out->status = st;
        return st;
    }

    std::vector<double> x(nf), g, sint(nf);
    for (int i = 0; i < nf; ++i) {
        x[i] = P.to_int(i, theta0[P.idx[i]]);
        double J = fabs(P.jac(i, x[i]));
        sint[i] = s0[i] / std::max(J, 1e-8);
        if (P.bounded[P.idx[i]]) sint[i] = std::min(sint[i], 0.5);
    }
    if (opt.strategy == 4) return newton_minimise(P, *hess, opt, x, sint, theta0, out);

    double f;
    int st = P.eval_int(x, f, g);
    if (st != NLL_OK) {
        out->status = st;
        out->n_eval = P.n_eval;
        return st;
    }

    // initial inverse Hessian
    std::vector<double> V((size_t)nf * nf, 0.0);
    auto diag_init = [&]() {
        std::fill(V.begin(), V.end(), 0.0);
        for (int i = 0; i < nf; ++i) V[i * nf + i] = sint[i] * sint[i];
    };
    // analytic second derivatives of the free parameters at external point th_free
    auto analytic_at = [&](const std::vector<double>& th_free, std::vector<double>& Hf,
                           std::vector<double>* Wf) -> bool {
        std::vector<double> th = P.base, Hn((size_t)n * n), Wn;
        for (int i = 0; i < nf; ++i) th[P.idx[i]] = th_free[i];
        if (Wf) Wn.resize((size_t)n * n);
        ++P.n_eval;
        double fh;
        std::vector<double> gh(n);
        if ((*hess)(th.data(), &fh, gh.data(), Hn.data(), Wf ? Wn.data() : nullptr) != NLL_OK) return false;
        Hf.resize((size_t)nf * nf);
        if (Wf) Wf->resize((size_t)nf * nf);
        for (int i = 0; i < nf; ++i)
            for (int j = 0; j < nf; ++j) {
                Hf[i * nf + j] = Hn[(size_t)P.idx[i] * n + P.idx[j]];
                if (Wf) (*Wf)[i * nf + j] = Wn[(size_t)P.idx[i] * n + P.idx[j]];
                if (!isfinite(Hf[i * nf + j])) return false;
            }
        return true;
    };
    diag_init();
    if (opt.strategy == 2) {
        // analytic Hessian in internal coordinates: J H J + diag(dF/dext d2ext/dx2)
        std::vector<double> th_free(nf), He;
        for (int i = 0; i < nf; ++i) th_free[i] = P.to_ext(i, x[i]);
        if (analytic_at(th_free, He, nullptr)) {
            std::vector<double> Hi((size_t)nf * nf), Vi((size_t)nf * nf);
            for (int i = 0; i < nf; ++i) {
                const double Ji = P.jac(i, x[i]);
                for (int j = 0; j < nf; ++j) Hi[i * nf + j] = Ji * He[i * nf + j] * P.jac(j, x[j]);
                const int k = P.idx[i];
                if (P.bounded[k] && fabs(Ji) > 1e-300)
                    Hi[i * nf + i] += (g[i] / Ji) * (-(P.hi[k] - P.lo[k]) * 0.5 * sin(x[i]));
            }
            if (spd_inverse(nf, Hi.data(), Vi.data())) V = Vi;
        }
    } else if (opt.strategy >= 1) {
        std::vector<double> h(nf), H;
        for (int i = 0; i < nf; ++i) h[i] = 0.1 * sint[i];
        auto gat = [&](int k, double dh, std::vector<double>& gg) {
            std::vector<double> xx = x;
            xx[k] += dh;
            double ff;
            return P.eval_int(xx, ff, gg) == NLL_OK;
        };
        if (fd_hessian(nf, h, gat, H)) {
            std::vector<double> Vi((size_t)nf * nf);
            if (spd_inverse(nf, H.data(), Vi.data())) V = Vi;
        }
    }

    std::vector<double> p(nf), xn(nf), gn, sv(nf), yv(nf), Vy(nf);
    double edm = 0.0;
    {
        std::vector<double> Vg;
        matvec(nf, V, g, Vg);
        edm = 0.5 * dot(g, Vg);
    }
    int iter = 0;
    bool converged = edm < opt.tol_edm;
    bool first_update = true;
    while (!converged && iter < opt.max_iter) {
        GBNLL_TRACE("quasi-Newton iteration");
        ++iter;
        matvec(nf, V, g, p);
        for (int i = 0; i < nf; ++i) p[i] = -p[i];
        double gp = dot(g, p);
        if (!(gp < 0.0)) {  // not a descent direction: restart from the diagonal
            diag_init();
            matvec(nf, V, g, p);
            for (int i = 0; i < nf; ++i) p[i] = -p[i];
            gp = dot(g, p);
            if (!(gp < 0.0)) break;
        }
        // line search
        const double c1 = 1e-4, c2 = 0.9;
        double alpha = 1.0, fn_ = 0.0;
        bool ok = false;
        double best_a = 0.0, best_f = f;
        std::vector<double> best_g;
        for (int ls = 0; ls < 40; ++ls) {
            for (int i = 0; i < nf; ++i) xn[i] = x[i] + alpha * p[i];
            int s2 = P.eval_int(xn, fn_, gn);
            if (s2 == NLL_OK && fn_ <= f + c1 * alpha * gp) {
                if (fn_ < best_f || !ok) {
                    best_a = alpha;
                    best_f = fn_;
                    best_g = gn;
                }
                ok = true;
                double gnp = dot(gn, p);
                if (gnp < c2 * gp && alpha < 16.0 && ls < 6) {  // still steep: extrapolate
                    alpha *= 2.0;
                    continue;
                }
                break;
            }
            if (ok) break;  // an extrapolation overshot: keep the best accepted point
            double anew;
            if (s2 == NLL_OK && isfinite(fn_)) {
                // minimiser of the quadratic through f, gp, fn_
                double denom = 2.0 * (fn_ - f - gp * alpha);
                anew = denom > 0.0 ? -gp * alpha * alpha / denom : 0.5 * alpha;
                anew = std::min(std::max(anew, 0.1 * alpha), 0.5 * alpha);
            } else {
                anew = 0.25 * alpha;
            }
            alpha = anew;
        }
        if (!ok) break;  // no decrease possible along p
        alpha = best_a;
        for (int i = 0; i < nf; ++i) {
            xn[i] = x[i] + alpha * p[i];
            sv[i] = xn[i] - x[i];
            yv[i] = best_g[i] - g[i];
        }
        double ys = dot(yv, sv);
        double fprev = f;
        x = xn;
        f = best_f;
        g = best_g;
        if (ys > 1e-300 && ys > 1e-12 * sqrt(dot(yv, yv) * dot(sv, sv))) {
            if (first_update && opt.strategy < 1) {  // scale the initial matrix (Nocedal & Wright 6.20)
                double sc = ys / dot(yv, yv);
                std::fill(V.begin(), V.end(), 0.0);
                for (int i = 0; i < nf; ++i) V[i * nf + i] = sc;
            }
            first_update = false;
            matvec(nf, V, yv, Vy);
            double yVy = dot(yv, Vy);
            double rho = 1.0 / ys;
            for (int i = 0; i < nf; ++i)
                for (int j = 0; j < nf; ++j)
                    V[i * nf + j] += rho * ((1.0 + rho * yVy) * sv[i] * sv[j] - Vy[i] * sv[j] - sv[i] * Vy[j]);
        }
        std::vector<double> Vg;
        matvec(nf, V, g, Vg);
        edm = 0.5 * dot(g, Vg);
        converged = edm < opt.tol_edm;
        if (!converged && fprev - f <= 0.0 && iter > 2) break;
    }

    // external free parameters and the quasi-Newton covariance
    std::vector<double> th_free(nf), J(nf);
    for (int i = 0; i < nf; ++i) {
        th_free[i] = P.to_ext(i, x[i]);
        J[i] = P.jac(i, x[i]);
    }
    std::vector<double> C((size_t)nf * nf);
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nf; ++j) C[i * nf + j] = J[i] * V[i * nf + j] * J[j];

    if (opt.hessian >= 1) {
        // FD Hessian of the analytic gradient in external coordinates, Newton polish
        std::vector<double> ge, H;
        double fe;
        int s3 = P.eval_ext(th_free, fe, ge);
        if (s3 == NLL_OK) {
            std::vector<double> h(nf);
            for (int i = 0; i < nf; ++i) {
                double sd = sqrt(std::max(C[i * nf + i], 0.0));
                if (!(sd > 0.0)) sd = s0[i];
                h[i] = 1e-3 * sd;
            }
            for (int pol = 0; pol < 4; ++pol) {
                auto gat = [&](int k, double dh, std::vector<double>& gg) {
                    std::vector<double> t = th_free;
                    t[k] += dh;
                    double ff;
                    return P.eval_ext(t, ff, gg) == NLL_OK;
                };
                if (opt.hessian >= 2 ? !analytic_at(th_free, H, nullptr) : !fd_hessian(nf, h, gat, H)) break;
                std::vector<double> Hi((size_t)nf * nf);
                if (!spd_inverse(nf, H.data(), Hi.data())) break;
                C = Hi;
                std::vector<double> d;
                matvec(nf, Hi, ge, d);
                edm = 0.5 * dot(ge, d);
                converged = edm < opt.tol_edm;
                if (converged) break;
                // Newton step (halved until it decreases and stays inside the bounds)
                double lam = 1.0;
                bool took = false;
                for (int t = 0; t < 20; ++t) {
                    std::vector<double> trial(nf);
                    bool inside = true;
                    for (int i = 0; i < nf; ++i) {
                        trial[i] = th_free[i] - lam * d[i];
                        int k = P.idx[i];
                        if (P.bounded[k] && (trial[i] <= P.lo[k] || trial[i] >= P.hi[k])) inside = false;
                    }
                    if (inside) {
                        std::vector<double> gt;
                        double ft;
                        if (P.eval_ext(trial, ft, gt) == NLL_OK && ft <= fe + 1e-15 * fabs(fe)) {
                            th_free = trial;
                            fe = ft;
                            ge = gt;
                            took = true;
                            break;
                        }
                    }
                    lam *= 0.5;
                }
                if (!took) break;
                for (int i = 0; i < nf; ++i) h[i] = 1e-3 * sqrt(std::max(C[i * nf + i], 1e-300));
            }
            if (opt.hessian >= 2) {
                // covariance at the final point: H^-1, or H^-1 W H^-1 for weighted fits
                std::vector<double> Wf, Hi((size_t)nf * nf);
                if (analytic_at(th_free, H, opt.hessian == 3 ? &Wf : nullptr) && spd_inverse(nf, H.data(), Hi.data())) {
                    if (opt.hessian == 3) {
                        std::vector<double> T((size_t)nf * nf, 0.0);
                        for (int i = 0; i < nf; ++i)
                            for (int k = 0; k < nf; ++k)
                                for (int j = 0; j < nf; ++j) T[i * nf + j] += Hi[i * nf + k] * Wf[k * nf + j];
                        for (int i = 0; i < nf; ++i)
                            for (int j = 0; j < nf; ++j) {
                                double sacc = 0.0;
                                for (int k = 0; k < nf; ++k) sacc += T[i * nf + k] * Hi[k * nf + j];
                                C[i * nf + j] = sacc;
                            }
                    } else {
                        C = Hi;
                    }
                    std::vector<double> d;
                    matvec(nf, Hi, ge, d);
                    edm = 0.5 * dot(ge, d);
                    converged = edm < opt.tol_edm;
                } else {
                    converged = false;
                }
            } else if (!converged) {
                std::vector<double> d;
                matvec(nf, C, ge, d);
                edm = 0.5 * dot(ge, d);
                converged = edm < opt.tol_edm;
            }
            f = fe;
        }
    }

    for (int k = 0; k < n; ++k) out->theta[k] = theta0[k];
    for (int i = 0; i < nf; ++i) out->theta[P.idx[i]] = th_free[i];
    for (int i = 0; i < nf; ++i) {
        for (int j = 0; j < nf; ++j) out->cov[P.idx[i] * n + P.idx[j]] = C[i * nf + j];
        out->err[P.idx[i]] = sqrt(std::max(C[i * nf + i], 0.0));
    }
    out->nll = f;
    out->edm = edm;
    out->n_eval = P.n_eval;
    out->n_iter = iter;
    out->status = converged ? NLL_OK : NLL_ERR_NOT_CONVERGED;
    return out->status;
}

}  // namespace gbnll

extern "C" int fit_minimise_fcn(fit_fcn fcn, void* user, const double* theta0, const double* lo, const double* hi,
                                const double* step, const int* fixed, int n_params, const fit_options* opt,
                                fit_result* out)
{
    if (!fcn || !out) return NLL_ERR_ARG;
    if (opt && (opt->strategy == 2 || opt->strategy == 4 || opt->hessian >= 2)) {  // needs second derivatives
        memset(out, 0, sizeof(*out));
        out->status = NLL_ERR_ARG;
        return NLL_ERR_ARG;
    }
    gbnll::Objective obj = [&](const double* th, double* f, double* g) {
        return fcn(user, th, f, g) == 0 ? (int)NLL_OK : (int)NLL_ERR_ARG;
    };
    return gbnll::bfgs_minimise(obj, n_params, theta0, lo, hi, step, fixed, opt, out);
}
