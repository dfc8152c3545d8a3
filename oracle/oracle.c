/*
 * oracle.c -- plain, slow CPU reference for the unbinned negative log-likelihood
 * of arXiv 2505.12414 (MoreFit) and its gradient, in IEEE FP64 with Kahan summation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent oracle that the CUDA path
 * is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load it.  It shares no code, header, table or constant with the
 * CUDA library, and it never calls it.
 *
 * What it computes (paper Sec. 2.1, Eq. 1):
 *     NLL(theta) = - sum_i w_i ln P(x_i | theta)
 * with w_i = 1 unless weights are given, and the gradient dNLL/dtheta from
 * hand-derived per-parameter derivatives of P (paper Sec. 2.1 asks for analytic
 * first derivatives; it does not print them).  Every event term is evaluated from
 * the plain definition of the model -- no hoisting, no precomputation, no
 * log-sum-exp -- and summed in event order with Kahan's compensated summation
 * (paper Sec. 2.3.1 / 2.3.2 use Kahan summation on host and accelerator).
 *
 * Models
 *   kind 1, mass model (paper Sec. 2.4.1, Eq. 2), theta = [mu, sigma, alpha, fsig]:
 *     P(m) = fsig * G(m) + (1 - fsig) * E(m)
 *     G(m) = exp(-(m-mu)^2 / (2 sigma^2)) / (sqrt(2 pi) sigma N1)
 *     N1   = 1/2 [erf((mu-ma)/(sqrt2 sigma)) - erf((mu-mb)/(sqrt2 sigma))]
 *     E(m) = exp(alpha m) / N2,  N2 = integral_{ma}^{mb} exp(alpha m) dm
 *            = (exp(alpha mb) - exp(alpha ma)) / alpha, and mb - ma at alpha == 0.
 *     N2 is evaluated as exp(alpha ma) expm1(alpha (mb-ma)) / alpha, the same
 *     integral written without the cancellation of the two exponentials.
 *   kind 2, four-dimensional B0 -> K*0 mu mu model, observables (m, cos theta_l,
 *     cos theta_K, phi), theta = [mu, sigma, FL, S3, S4, S5, AFB, S7, S8, S9,
 *     alpha, c1_l, c2_l, c1_K, c2_K, c1_phi, c2_phi, fsig]:
 *     P = fsig G(m) A(ctl,ctk,phi) + (1-fsig) E(m) prod_j C_j(x_j)/Nc_j
 *     A is the angular decay rate of paper Sec. 2.4.2, Eq. 3 (eleven terms, with
 *     the overall 9/(32 pi)), integrating to 1 over ctl, ctk in [-1,1] and phi in
 *     [-pi, pi].  sin theta = +sqrt(1 - cos^2 theta), sin 2t = 2 sin t cos t and
 *     cos 2t = 2 cos^2 t - 1.
 *     C_j(x) = 1 + c1_j x + c2_j (2 x^2 - 1) (second-order Chebyshev series with the
 *     T0 coefficient fixed to one) in x_1 = ctl, x_2 = ctk, x_3 = phi/pi; Nc_j is its
 *     integral over the observable: 2 - (2/3) c2 in ctl and ctk, pi (2 - (2/3) c2)
 *     in phi.  The paper has no background model for its angular fit; this
 *     exponential-times-Chebyshev background is the reading taken for the 4D
 *     benchmark configuration.
 *
 * Second derivatives (paper Sec. 2.1 names the analytic Hessian used for the HESSE
 * uncertainties, and the Fisher information needed for weighted fits, without printing
 * either): oracle_nll_hess returns
 *     H_ab = d^2 NLL / dtheta_a dtheta_b = - sum_i w_i (P_ab / P - P_a P_b / P^2)_i
 *     W_ab = sum_i w_i^2 (P_a / P)_i (P_b / P)_i
 * from hand-derived second derivatives P_ab of the plain model.  For a weighted fit the
 * asymptotic covariance is H^-1 W H^-1 (Langenbruch, Eur. Phys. J. C 82 (2022) 393, the
 * reference the paper gives for weighted fits); for w = 1 both H and W estimate the
 * Fisher information.
 *
 * Threads: events are split into static contiguous chunks, each chunk sums with
 * Kahan, and the chunk sums are merged in chunk order (again with Kahan), so the
 * result does not depend on scheduling.  The chunks run on worker threads started at
 * the first multi-threaded call and kept until the process exits.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NONPOSITIVE 4

#define OR_MASS1D 1
#define OR_KSTAR4D 2

#define OR_MAXPAR 18

static const double kPi = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Kahan's compensated summation (paper cites Kahan 1965).            */
/* ------------------------------------------------------------------ */
typedef struct {
    double s, c;
} kahan_t;

static void kahan_add(kahan_t* k, double x)
{
    double y = x - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* ------------------------------------------------------------------ */
/* Mass part: normalisations of paper Eq. 2 and their derivatives.    */
/* ------------------------------------------------------------------ */
typedef struct {
    double ma, mb;
    double mu, sigma, alpha;
    double N1;          /* Gaussian normalisation over [ma, mb]                     */
    double dlnN1_dmu;   /* d ln N1 / d mu                                           */
    double dlnN1_dsig;  /* d ln N1 / d sigma                                        */
    double N2;          /* exponential normalisation over [ma, mb]                  */
    double dlnN2_dal;   /* d ln N2 / d alpha                                        */
    double d2lnN1[3];   /* d^2 ln N1 / (dmu dmu, dmu dsigma, dsigma dsigma)          */
    double d2lnN2_dal2; /* d^2 ln N2 / d alpha^2 = (mb - ma)^2 v(alpha (mb - ma))    */
} mass_norm_t;

static void mass_norm(mass_norm_t* n, double ma, double mb, double mu, double sigma, double alpha)
{
    n->ma = ma;
    n->mb = mb;
    n->mu = mu;
    n->sigma = sigma;
    n->alpha = alpha;
    /* N1 = 1/2 [erf(za) - erf(zb)], za = (mu-ma)/(sqrt2 sigma), zb = (mu-mb)/(sqrt2 sigma) */
    double za = (mu - ma) / (sqrt(2.0) * sigma);
    double zb = (mu - mb) / (sqrt(2.0) * sigma);
    n->N1 = 0.5 * (erf(za) - erf(zb));
    /* d erf(z)/dz = 2/sqrt(pi) exp(-z^2);  dza/dmu = 1/(sqrt2 sigma);  dza/dsigma = -za/sigma */
    double ea = exp(-za * za), eb = exp(-zb * zb);
    double dN1_dmu = (ea - eb) / (sqrt(2.0 * kPi) * sigma);
    double dN1_dsig = -(za * ea - zb * eb) / (sqrt(kPi) * sigma);
    n->dlnN1_dmu = dN1_dmu / n->N1;
    n->dlnN1_dsig = dN1_dsig / n->N1;
    /* second derivatives of N1: differentiate the two first derivatives above once more,
     * with d ea / dmu = -2 za ea / (sqrt2 sigma) and d ea / dsigma = 2 za^2 ea / sigma */
    double d2N1_mumu = -(za * ea - zb * eb) / (sqrt(kPi) * sigma * sigma);
    double d2N1_musig = (ea * (2.0 * za * za - 1.0) - eb * (2.0 * zb * zb - 1.0)) / (sqrt(2.0 * kPi) * sigma * sigma);
    double d2N1_sigsig = (za * ea * (2.0 - 2.0 * za * za) - zb * eb * (2.0 - 2.0 * zb * zb)) / (sqrt(kPi) * sigma * sigma);
    /* d^2 ln N = N''/N - (N'/N)(N'/N) */
    n->d2lnN1[0] = d2N1_mumu / n->N1 - n->dlnN1_dmu * n->dlnN1_dmu;
    n->d2lnN1[1] = d2N1_musig / n->N1 - n->dlnN1_dmu * n->dlnN1_dsig;
    n->d2lnN1[2] = d2N1_sigsig / n->N1 - n->dlnN1_dsig * n->dlnN1_dsig;
    /* N2 = integral exp(alpha m) dm over [ma, mb]; the paper's alpha == 0 branch gives mb - ma */
    double D = mb - ma;
    /* d^2 ln N2 / d alpha^2 is the variance of m under exp(alpha m) on [ma, mb]:
     * D^2 v(t), t = alpha D, v(t) = 1/t^2 - e^t / (e^t - 1)^2 = 1/t^2 - 1/(4 sinh^2(t/2)),
     * even in t, v(0) = 1/12 (uniform).  From the series of coth,
     *   v(t) = sum_{n >= 1} (2n - 1) B_2n t^(2n-2) / (2n)!   (|t| < 2 pi),
     * used for |t| < 1/2 with n <= 9 (next term below 1e-18 of v there); above, the closed
     * form loses at most ~12 u / t^2 to cancellation, written with e^-|t| so it cannot overflow. */
    {
        static const double bern[10] = {0.0,          1.0 / 6.0,   -1.0 / 30.0,   1.0 / 42.0,      -1.0 / 30.0,
                                         5.0 / 66.0,   -691.0 / 2730.0, 7.0 / 6.0, -3617.0 / 510.0, 43867.0 / 798.0};
        double a = fabs(alpha * D), v;
        if (a < 0.5) {
            double t2 = a * a, fact = 2.0;  /* (2n)! */
            double coef[10];
            for (int k = 1; k <= 9; ++k) {
                if (k > 1) fact *= (2.0 * k - 1.0) * (2.0 * k);
                coef[k] = (2.0 * k - 1.0) * bern[k] / fact;
            }
            v = coef[9];
            for (int k = 8; k >= 1; --k) v = v * t2 + coef[k];
        } else {
            double em = expm1(-a);
            v = 1.0 / (a * a) - exp(-a) / (em * em);
        }
        n->d2lnN2_dal2 = D * D * v;
    }
    if (alpha == 0.0) {
        n->N2 = D;
        n->dlnN2_dal = 0.5 * (ma + mb);
    } else {
        n->N2 = exp(alpha * ma) * expm1(alpha * D) / alpha;
        double t = alpha * D;
        if (fabs(t) > 1e-3) {
            /* d ln N2/d alpha = ma + D e^t/(e^t - 1) - 1/alpha */
            n->dlnN2_dal = ma + D * exp(t) / expm1(t) - 1.0 / alpha;
        } else {
            /* same quantity from the series 1/(1-e^-t) - 1/t = 1/2 + t/12 - t^3/720 + t^5/30240 */
            double t2 = t * t;
            n->dlnN2_dal = ma + D * (0.5 + t / 12.0 - t * t2 / 720.0 + t * t2 * t2 / 30240.0);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Angular part: the eleven terms of paper Eq. 3.                      */
/*   A = sum_i S_i f_i,  S = [1-FL, FL, 1-FL, -FL, S3, S4, S5, AFB,    */
/*                            S7, S8, S9]                              */
/* f_i already carries the overall 9/(32 pi).                          */
/* ------------------------------------------------------------------ */
static void angular_terms(double ctl, double ctk, double phi, double f[11])
{
    const double c = 9.0 / (32.0 * kPi);
    double sl2 = 1.0 - ctl * ctl, sk2 = 1.0 - ctk * ctk;
    double sl = sqrt(sl2), sk = sqrt(sk2);
    double cl2 = ctl * ctl, ck2 = ctk * ctk;
    double cos2l = 2.0 * cl2 - 1.0;
    double sin2l = 2.0 * sl * ctl, sin2k = 2.0 * sk * ctk;
    double cphi = cos(phi), sphi = sin(phi), c2phi = cos(2.0 * phi), s2phi = sin(2.0 * phi);
    f[0] = c * 0.75 * sk2;                  /* (1-FL) 3/4 sin^2 tK              */
    f[1] = c * ck2;                         /* FL cos^2 tK                      */
    f[2] = c * 0.25 * sk2 * cos2l;          /* (1-FL) 1/4 sin^2 tK cos 2tl      */
    f[3] = c * ck2 * cos2l;                 /* -FL cos^2 tK cos 2tl             */
    f[4] = c * sk2 * sl2 * c2phi;           /* S3 sin^2 tK sin^2 tl cos 2phi     */
    f[5] = c * sin2k * sin2l * cphi;        /* S4 sin 2tK sin 2tl cos phi        */
    f[6] = c * sin2k * sl * cphi;           /* S5 sin 2tK sin tl cos phi         */
    f[7] = c * (4.0 / 3.0) * sk2 * ctl;     /* AFB 4/3 sin^2 tK cos tl           */
    f[8] = c * sin2k * sl * sphi;           /* S7 sin 2tK sin tl sin phi         */
    f[9] = c * sin2k * sin2l * sphi;        /* S8 sin 2tK sin 2tl sin phi        */
    f[10] = c * sk2 * sl2 * s2phi;          /* S9 sin^2 tK sin^2 tl sin 2phi     */
}

/* coefficients S_i(theta) of Eq. 3 and dS_i/d(FL, S3, S4, S5, AFB, S7, S8, S9) */
static void angular_coefs(const double* ang /* FL,S3,S4,S5,AFB,S7,S8,S9 */, double S[11])
{
    double FL = ang[0];
    S[0] = 1.0 - FL;
    S[1] = FL;
    S[2] = 1.0 - FL;
    S[3] = -FL;
    for (int k = 1; k < 8; ++k) S[3 + k] = ang[k];
}

/* ------------------------------------------------------------------ */
/* Per-event density and its parameter derivatives, plain definition. */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind;
    int npar;
    double ranges[8];
    double theta[OR_MAXPAR];
    mass_norm_t mn;
    double Nc[3];       /* Chebyshev normalisations (ctl, ctk, phi)    */
    double dNc_dc2[3];  /* dNc_j / dc2_j                                */
} model_t;

static int npar_of(int kind) { return kind == OR_MASS1D ? 4 : (kind == OR_KSTAR4D ? 18 : -1); }

static int model_setup(model_t* M, int kind, const double* ranges, const double* theta)
{
    int np = npar_of(kind);
    if (np < 0) return OR_ERR_ARG;
    M->kind = kind;
    M->npar = np;
    int nr = kind == OR_MASS1D ? 2 : 8;
    memcpy(M->ranges, ranges, sizeof(double) * nr);
    memcpy(M->theta, theta, sizeof(double) * np);
    double ma = ranges[0], mb = ranges[1];
    if (kind == OR_MASS1D) {
        /* theta = [mu, sigma, alpha, fsig] */
        mass_norm(&M->mn, ma, mb, theta[0], theta[1], theta[2]);
    } else {
        /* theta = [mu, sigma, FL..S9 (8), alpha, c1l, c2l, c1k, c2k, c1p, c2p, fsig] */
        mass_norm(&M->mn, ma, mb, theta[0], theta[1], theta[10]);
        for (int j = 0; j < 3; ++j) {
            double c2 = theta[12 + 2 * j];
            double scale = (j == 2) ? kPi : 1.0; /* dphi = pi dx */
            M->Nc[j] = scale * (2.0 - (2.0 / 3.0) * c2);
            M->dNc_dc2[j] = scale * (-2.0 / 3.0);
        }
    }
    return OR_OK;
}

/* density of the Gaussian and exponential mass components and d ln / d(params) */
static void mass_parts(const mass_norm_t* n, double m, double* G, double* dlnG_dmu, double* dlnG_dsig,
                       double* E, double* dlnE_dal)
{
    double d = m - n->mu, s = n->sigma;
    *G = exp(-d * d / (2.0 * s * s)) / (sqrt(2.0 * kPi) * s * n->N1);
    *dlnG_dmu = d / (s * s) - n->dlnN1_dmu;
    *dlnG_dsig = d * d / (s * s * s) - 1.0 / s - n->dlnN1_dsig;
    *E = exp(n->alpha * m) / n->N2;
    *dlnE_dal = m - n->dlnN2_dal;
}

/* P and dP/dtheta for one event; returns P */
static double event_density(const model_t* M, const double* x, double* dP)
{
    const double* th = M->theta;
    double G, dGmu, dGsig, E, dEal;
    mass_parts(&M->mn, x[0], &G, &dGmu, &dGsig, &E, &dEal);
    if (M->kind == OR_MASS1D) {
        double f = th[3];
        double P = f * G + (1.0 - f) * E;
        if (dP) {
            dP[0] = f * G * dGmu;
            dP[1] = f * G * dGsig;
            dP[2] = (1.0 - f) * E * dEal;
            dP[3] = G - E;
        }
        return P;
    }
    /* 4D */
    double fa[11], S[11];
    angular_terms(x[1], x[2], x[3], fa);
    angular_coefs(th + 2, S);
    double A = 0.0;
    for (int i = 0; i < 11; ++i) A += S[i] * fa[i];
    double xs[3] = {x[1], x[2], x[3] / kPi};
    double Cn[3];  /* C_j / Nc_j */
    for (int j = 0; j < 3; ++j) {
        double c1 = th[11 + 2 * j], c2 = th[12 + 2 * j];
        double xv = xs[j];
        double Cj = 1.0 + c1 * xv + c2 * (2.0 * xv * xv - 1.0);
        Cn[j] = Cj / M->Nc[j];
    }
    double B = Cn[0] * Cn[1] * Cn[2];
    double f = th[17];
    double P = f * G * A + (1.0 - f) * E * B;
    if (dP) {
        dP[0] = f * A * G * dGmu;
        dP[1] = f * A * G * dGsig;
        /* dA/dFL = -f0 + f1 - f2 - f3 ; dA/dS_k = f_(3+k) */
        dP[2] = f * G * (-fa[0] + fa[1] - fa[2] - fa[3]);
        for (int k = 1; k < 8; ++k) dP[2 + k] = f * G * fa[3 + k];
        dP[10] = (1.0 - f) * E * dEal * B;
        for (int j = 0; j < 3; ++j) {
            double others = 1.0;
            for (int k = 0; k < 3; ++k)
                if (k != j) others *= Cn[k];
            double xv = xs[j];
            double T2 = 2.0 * xv * xv - 1.0;
            double c1 = th[11 + 2 * j], c2 = th[12 + 2 * j];
            double Cj = 1.0 + c1 * xv + c2 * T2;
            /* d(Cj/Nc)/dc1 = x/Nc ; d(Cj/Nc)/dc2 = T2/Nc - Cj dNc/dc2 / Nc^2 */
            double dc1 = xv / M->Nc[j];
            double dc2 = T2 / M->Nc[j] - Cj * M->dNc_dc2[j] / (M->Nc[j] * M->Nc[j]);
            dP[11 + 2 * j] = (1.0 - f) * E * others * dc1;
            dP[12 + 2 * j] = (1.0 - f) * E * others * dc2;
        }
        dP[17] = G * A - E * B;
    }
    return P;
}

/* Second derivatives d2P[a * npar + b] = d^2 P / dtheta_a dtheta_b for one event, written
 * out from the plain definition of the model term by term (symmetric; unlisted pairs are 0). */
static void event_second(const model_t* M, const double* x, double* d2P)
{
    const double* th = M->theta;
    const int np = M->npar;
    memset(d2P, 0, sizeof(double) * np * np);
#define SET2(a, b, v)               \
    do {                            \
        double v_ = (v);            \
        d2P[(a) * np + (b)] = v_;   \
        d2P[(b) * np + (a)] = v_;   \
    } while (0)
    double G, dGmu, dGsig, E, dEal;
    mass_parts(&M->mn, x[0], &G, &dGmu, &dGsig, &E, &dEal);
    /* second log-derivatives of the Gaussian and of the exponential (paper Eq. 2):
     * ln G = -d^2/(2 s^2) - ln s - ln N1 + const,  ln E = alpha m - ln N2 */
    double d = x[0] - M->mn.mu, s = M->mn.sigma;
    double hmm = -1.0 / (s * s) - M->mn.d2lnN1[0];
    double hms = -2.0 * d / (s * s * s) - M->mn.d2lnN1[1];
    double hss = -3.0 * d * d / (s * s * s * s) + 1.0 / (s * s) - M->mn.d2lnN1[2];
    double haa = -M->mn.d2lnN2_dal2;
    /* d^2 G / da db = G (dlnG/da dlnG/db + d^2 lnG / da db), likewise for E */
    double Gmm = G * (dGmu * dGmu + hmm), Gms = G * (dGmu * dGsig + hms), Gss = G * (dGsig * dGsig + hss);
    double Eaa = E * (dEal * dEal + haa);
    if (M->kind == OR_MASS1D) {
        /* P = f G + (1 - f) E, theta = [mu, sigma, alpha, f] */
        double f = th[3];
        SET2(0, 0, f * Gmm);
        SET2(0, 1, f * Gms);
        SET2(1, 1, f * Gss);
        SET2(2, 2, (1.0 - f) * Eaa);
        SET2(3, 0, G * dGmu);
        SET2(3, 1, G * dGsig);
        SET2(3, 2, -E * dEal);
        return;
    }
    /* 4D: P = f G A + (1 - f) E B;  A linear in (FL, S3..S9), so d^2 A = 0 */
    double fa[11], S[11];
    angular_terms(x[1], x[2], x[3], fa);
    angular_coefs(th + 2, S);
    double A = 0.0;
    for (int i = 0; i < 11; ++i) A += S[i] * fa[i];
    double dA[8];
    dA[0] = -fa[0] + fa[1] - fa[2] - fa[3];
    for (int k = 1; k < 8; ++k) dA[k] = fa[3 + k];
    /* Chebyshev factors Cn_j = C_j / Nc_j and their derivatives in (c1_j, c2_j):
     *   dCn/dc1 = x/Nc, dCn/dc2 = T2/Nc - C Nc'/Nc^2,
     *   d2Cn/dc1^2 = 0, d2Cn/dc1dc2 = -x Nc'/Nc^2, d2Cn/dc2^2 = -2 T2 Nc'/Nc^2 + 2 C Nc'^2/Nc^3 */
    double xs[3] = {x[1], x[2], x[3] / kPi};
    double Cn[3], dCn[3][2], d2Cn[3][2][2];
    for (int j = 0; j < 3; ++j) {
        double c1 = th[11 + 2 * j], c2 = th[12 + 2 * j];
        double xv = xs[j], T2 = 2.0 * xv * xv - 1.0;
        double Cj = 1.0 + c1 * xv + c2 * T2;
        double Nc = M->Nc[j], Np = M->dNc_dc2[j];
        Cn[j] = Cj / Nc;
        dCn[j][0] = xv / Nc;
        dCn[j][1] = T2 / Nc - Cj * Np / (Nc * Nc);
        d2Cn[j][0][0] = 0.0;
        d2Cn[j][0][1] = d2Cn[j][1][0] = -xv * Np / (Nc * Nc);
        d2Cn[j][1][1] = -2.0 * T2 * Np / (Nc * Nc) + 2.0 * Cj * Np * Np / (Nc * Nc * Nc);
    }
    double B = Cn[0] * Cn[1] * Cn[2];
    /* B derivatives: index 2 j + p for coefficient p (0: c1, 1: c2) of observable j */
    double dB[6], d2B[6][6];
    for (int j = 0; j < 3; ++j) {
        double others = 1.0;
        for (int k = 0; k < 3; ++k)
            if (k != j) others *= Cn[k];
        for (int p = 0; p < 2; ++p) dB[2 * j + p] = others * dCn[j][p];
    }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) {
                    double v;
                    if (j == k) {
                        double others = 1.0;
                        for (int l = 0; l < 3; ++l)
                            if (l != j) others *= Cn[l];
                        v = others * d2Cn[j][p][q];
                    } else {
                        double third = 1.0;
                        for (int l = 0; l < 3; ++l)
                            if (l != j && l != k) third *= Cn[l];
                        v = third * dCn[j][p] * dCn[k][q];
                    }
                    d2B[2 * j + p][2 * k + q] = v;
                }
    double f = th[17];
    /* signal block: mass x mass, mass x angular (angular x angular is zero) */
    SET2(0, 0, f * A * Gmm);
    SET2(0, 1, f * A * Gms);
    SET2(1, 1, f * A * Gss);
    for (int k = 0; k < 8; ++k) {
        SET2(0, 2 + k, f * G * dGmu * dA[k]);
        SET2(1, 2 + k, f * G * dGsig * dA[k]);
    }
    /* background block: alpha x alpha, alpha x Chebyshev, Chebyshev x Chebyshev */
    SET2(10, 10, (1.0 - f) * Eaa * B);
    for (int i = 0; i < 6; ++i) SET2(10, 11 + i, (1.0 - f) * E * dEal * dB[i]);
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) SET2(11 + i, 11 + j, (1.0 - f) * E * d2B[i][j]);
    /* signal fraction: d/df of the first derivatives (d^2 P / df^2 = 0) */
    SET2(17, 0, A * G * dGmu);
    SET2(17, 1, A * G * dGsig);
    for (int k = 0; k < 8; ++k) SET2(17, 2 + k, G * dA[k]);
    SET2(17, 10, -E * dEal * B);
    for (int i = 0; i < 6; ++i) SET2(17, 11 + i, -E * dB[i]);
#undef SET2
}

/* ------------------------------------------------------------------ */
/* Worker threads, started once and kept for the life of the process, */
/* so that a call's time is its arithmetic and not thread start-up.   */
/* A call hands chunk t (t >= 1) to worker t-1 and runs chunk 0       */
/* itself; which thread runs a chunk does not change any result,      */
/* since every chunk is summed on its own and merged in chunk order.  */
/* ------------------------------------------------------------------ */
#define OR_POOL_MAX 256

typedef struct {
    pthread_mutex_t mu;       /* guards everything below                        */
    pthread_cond_t go, done;  /* new work published / a worker finished         */
    pthread_mutex_t call_mu;  /* one call at a time uses the workers             */
    int nworkers;
    unsigned long gen;        /* incremented for every call's work               */
    int pending;              /* chunks handed out and not yet finished          */
    int ntasks;               /* chunks of the current call (chunk 0: the caller) */
    void* (*fn)(void*);
    char* args;
    size_t stride;
} pool_t;

static pool_t g_pool = {PTHREAD_MUTEX_INITIALIZER, PTHREAD_COND_INITIALIZER, PTHREAD_COND_INITIALIZER,
                        PTHREAD_MUTEX_INITIALIZER, 0, 0, 0, 0, NULL, NULL, 0};
/* generation counter at each worker's creation: work published after it is the worker's */
static unsigned long g_worker_gen0[OR_POOL_MAX];
static pthread_once_t g_pool_once = PTHREAD_ONCE_INIT;

static void* pool_worker(void* arg)
{
    const int id = (int)(intptr_t)arg; /* runs chunk id + 1 */
    pthread_mutex_lock(&g_pool.mu);
    unsigned long seen = g_worker_gen0[id];
    for (;;) {
        while (g_pool.gen == seen) pthread_cond_wait(&g_pool.go, &g_pool.mu);
        seen = g_pool.gen;
        if (id + 1 >= g_pool.ntasks) continue;
        void* (*fn)(void*) = g_pool.fn;
        void* a = g_pool.args + (size_t)(id + 1) * g_pool.stride;
        pthread_mutex_unlock(&g_pool.mu);
        fn(a);
        pthread_mutex_lock(&g_pool.mu);
        if (--g_pool.pending == 0) pthread_cond_signal(&g_pool.done);
    }
    return NULL;
}

/* A child made by fork() has none of the parent's worker threads: forget them there. */
static void pool_after_fork_child(void)
{
    pthread_mutex_init(&g_pool.mu, NULL);
    pthread_cond_init(&g_pool.go, NULL);
    pthread_cond_init(&g_pool.done, NULL);
    pthread_mutex_init(&g_pool.call_mu, NULL);
    g_pool.nworkers = 0;
    g_pool.pending = 0;
    g_pool.ntasks = 0;
}

static void pool_register_fork(void) { pthread_atfork(NULL, NULL, pool_after_fork_child); }

/* Run fn on ntasks argument blocks (args + t * stride); returns once all have finished.
 * Falls back to running everything on the calling thread if workers cannot be started. */
static void pool_run(void* (*fn)(void*), void* args, size_t stride, int ntasks)
{
    char* base = (char*)args;
    if (ntasks <= 1) {
        if (ntasks == 1) fn(base);
        return;
    }
    pthread_once(&g_pool_once, pool_register_fork);
    pthread_mutex_lock(&g_pool.call_mu);
    pthread_mutex_lock(&g_pool.mu);
    while (g_pool.nworkers < ntasks - 1 && g_pool.nworkers < OR_POOL_MAX - 1) {
        pthread_t t;
        g_worker_gen0[g_pool.nworkers] = g_pool.gen;
        if (pthread_create(&t, NULL, pool_worker, (void*)(intptr_t)g_pool.nworkers) != 0) break;
        pthread_detach(t);
        g_pool.nworkers++;
    }
    int nw = g_pool.nworkers < ntasks - 1 ? g_pool.nworkers : ntasks - 1;
    g_pool.fn = fn;
    g_pool.args = base;
    g_pool.stride = stride;
    g_pool.ntasks = nw + 1;
    g_pool.pending = nw;
    g_pool.gen++;
    pthread_cond_broadcast(&g_pool.go);
    pthread_mutex_unlock(&g_pool.mu);
    fn(base);
    for (int t = nw + 1; t < ntasks; ++t) fn(base + (size_t)t * stride); /* chunks no worker took */
    pthread_mutex_lock(&g_pool.mu);
    while (g_pool.pending > 0) pthread_cond_wait(&g_pool.done, &g_pool.mu);
    pthread_mutex_unlock(&g_pool.mu);
    pthread_mutex_unlock(&g_pool.call_mu);
}

/* ------------------------------------------------------------------ */
/* Event loop with Kahan sums, split over threads in static chunks.   */
/* ------------------------------------------------------------------ */
typedef struct {
    const model_t* M;
    const double* const* cols;
    const double* w;
    int64_t lo, hi;
    int want_grad;
    kahan_t nll;
    kahan_t g[OR_MAXPAR];
    kahan_t sc[OR_MAXPAR];
    int64_t bad;
} chunk_t;

static void* chunk_run(void* arg)
{
    chunk_t* c = (chunk_t*)arg;
    const model_t* M = c->M;
    int ndim = M->kind == OR_MASS1D ? 1 : 4;
    int np = M->npar;
    double x[4], dP[OR_MAXPAR];
    for (int64_t i = c->lo; i < c->hi; ++i) {
        for (int d = 0; d < ndim; ++d) x[d] = c->cols[d][i];
        double wi = c->w ? c->w[i] : 1.0;
        double P = event_density(M, x, c->want_grad ? dP : NULL);
        if (!(P > 0.0) || !isfinite(P)) {
            c->bad++;
            continue;
        }
        kahan_add(&c->nll, -wi * log(P));
        if (c->want_grad) {
            for (int k = 0; k < np; ++k) {
                double t = wi * dP[k] / P;
                kahan_add(&c->g[k], -t);
                kahan_add(&c->sc[k], fabs(t));
            }
        }
    }
    return NULL;
}

/*
 * oracle_nll_grad: NLL, gradient and per-component scales S_k = sum_i |w_i dl_i/dtheta_k|.
 *   kind       1 (mass) or 2 (4D)
 *   ranges     [ma, mb] (kind 1) or [ma, mb, -1, 1, -1, 1, -pi, pi] (kind 2)
 *   cols       ndim pointers to host arrays of n doubles (m; or m, ctl, ctk, phi)
 *   w          per-event weights or NULL (all ones)
 *   theta      parameters (4 or 18)
 *   nthreads   >= 1
 *   grad,scale may be NULL (NLL only)
 * Returns OR_OK, or OR_ERR_NONPOSITIVE with *nll = +inf when some P_i <= 0 or is not finite.
 */
int oracle_nll_grad(int kind, const double* ranges, const double* const* cols, const double* w, int64_t n,
                    const double* theta, int nthreads, double* nll, double* grad, double* scale)
{
    model_t M;
    if (model_setup(&M, kind, ranges, theta) != OR_OK || n < 0 || nthreads < 1) return OR_ERR_ARG;
    int want_grad = grad != NULL;
    if (nthreads > 256) nthreads = 256;
    if (n < (int64_t)nthreads * 64) nthreads = 1;
    chunk_t* ch = (chunk_t*)calloc((size_t)nthreads, sizeof(chunk_t));
    if (!ch) return OR_ERR_ARG;
    for (int t = 0; t < nthreads; ++t) {
        ch[t].M = &M;
        ch[t].cols = cols;
        ch[t].w = w;
        ch[t].lo = n * t / nthreads;
        ch[t].hi = n * (t + 1) / nthreads;
        ch[t].want_grad = want_grad;
    }
    pool_run(chunk_run, ch, sizeof(chunk_t), nthreads);
    kahan_t tot = {0, 0}, g[OR_MAXPAR], sc[OR_MAXPAR];
    memset(g, 0, sizeof g);
    memset(sc, 0, sizeof sc);
    int64_t bad = 0;
    for (int t = 0; t < nthreads; ++t) {
        kahan_add(&tot, ch[t].nll.s);
        kahan_add(&tot, -ch[t].nll.c);
        for (int k = 0; k < M.npar; ++k) {
            kahan_add(&g[k], ch[t].g[k].s);
            kahan_add(&g[k], -ch[t].g[k].c);
            kahan_add(&sc[k], ch[t].sc[k].s);
            kahan_add(&sc[k], -ch[t].sc[k].c);
        }
        bad += ch[t].bad;
    }
    free(ch);
    if (bad) {
        *nll = INFINITY;
        return OR_ERR_NONPOSITIVE;
    }
    *nll = tot.s;
    if (want_grad)
        for (int k = 0; k < M.npar; ++k) grad[k] = g[k].s;
    if (scale)
        for (int k = 0; k < M.npar; ++k) scale[k] = sc[k].s;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Hessian of the NLL and the squared-weight score outer product.      */
/* ------------------------------------------------------------------ */
typedef struct {
    const model_t* M;
    const double* const* cols;
    const double* w;
    int64_t lo, hi;
    kahan_t nll;
    kahan_t g[OR_MAXPAR];
    kahan_t h[OR_MAXPAR * OR_MAXPAR];
    kahan_t hs[OR_MAXPAR * OR_MAXPAR];
    kahan_t w2[OR_MAXPAR * OR_MAXPAR];
    int64_t bad;
} hchunk_t;

static void* hchunk_run(void* arg)
{
    hchunk_t* c = (hchunk_t*)arg;
    const model_t* M = c->M;
    int ndim = M->kind == OR_MASS1D ? 1 : 4;
    int np = M->npar;
    double x[4], dP[OR_MAXPAR], d2P[OR_MAXPAR * OR_MAXPAR], sc[OR_MAXPAR];
    for (int64_t i = c->lo; i < c->hi; ++i) {
        for (int d = 0; d < ndim; ++d) x[d] = c->cols[d][i];
        double wi = c->w ? c->w[i] : 1.0;
        double P = event_density(M, x, dP);
        if (!(P > 0.0) || !isfinite(P)) {
            c->bad++;
            continue;
        }
        event_second(M, x, d2P);
        kahan_add(&c->nll, -wi * log(P));
        for (int a = 0; a < np; ++a) {
            sc[a] = dP[a] / P;
            kahan_add(&c->g[a], -(wi * dP[a] / P));  /* the same rounding as oracle_nll_grad */
        }
        for (int a = 0; a < np; ++a)
            for (int b = a; b < np; ++b) {
                /* d^2 ln P / da db = P_ab / P - (P_a / P)(P_b / P) */
                double q = d2P[a * np + b] / P, pp = sc[a] * sc[b];
                double t = wi * (q - pp);
                kahan_add(&c->h[a * np + b], -t);
                /* the two terms cancel where one mixture component dominates the event, so
                 * the rounding error of t is bounded by the size of the terms, not of t */
                kahan_add(&c->hs[a * np + b], fabs(wi) * (fabs(q) + fabs(pp)));
                kahan_add(&c->w2[a * np + b], wi * wi * sc[a] * sc[b]);
            }
    }
    return NULL;
}

/*
 * oracle_nll_hess: NLL, gradient, Hessian H of the NLL and W = sum_i w_i^2 s_i s_i^T
 * (s_i = d ln P_i / dtheta), all row-major npar x npar and symmetric, plus
 * hscale_ab = sum_i |w_i| (|P_ab / P| + |P_a P_b / P^2|)_i, the size of the two terms
 * whose difference makes up each event's share of H_ab (their cancellation, where one
 * mixture component dominates an event, is what limits this plain form's accuracy).
 * Arguments as oracle_nll_grad; grad, w2 and hscale may be NULL.  Status as there.
 */
int oracle_nll_hess(int kind, const double* ranges, const double* const* cols, const double* w, int64_t n,
                    const double* theta, int nthreads, double* nll, double* grad, double* hess, double* w2,
                    double* hscale)
{
    model_t M;
    if (model_setup(&M, kind, ranges, theta) != OR_OK || n < 0 || nthreads < 1 || !nll || !hess) return OR_ERR_ARG;
    if (nthreads > 256) nthreads = 256;
    if (n < (int64_t)nthreads * 64) nthreads = 1;
    hchunk_t* ch = (hchunk_t*)calloc((size_t)nthreads, sizeof(hchunk_t));
    if (!ch) return OR_ERR_ARG;
    for (int t = 0; t < nthreads; ++t) {
        ch[t].M = &M;
        ch[t].cols = cols;
        ch[t].w = w;
        ch[t].lo = n * t / nthreads;
        ch[t].hi = n * (t + 1) / nthreads;
    }
    pool_run(hchunk_run, ch, sizeof(hchunk_t), nthreads);
    const int np = M.npar;
    kahan_t tot = {0, 0};
    static const kahan_t zero = {0, 0};
    kahan_t g[OR_MAXPAR], h[OR_MAXPAR * OR_MAXPAR], hs[OR_MAXPAR * OR_MAXPAR], q[OR_MAXPAR * OR_MAXPAR];
    for (int k = 0; k < OR_MAXPAR; ++k) g[k] = zero;
    for (int k = 0; k < OR_MAXPAR * OR_MAXPAR; ++k) h[k] = hs[k] = q[k] = zero;
    int64_t bad = 0;
    for (int t = 0; t < nthreads; ++t) {
        kahan_add(&tot, ch[t].nll.s);
        kahan_add(&tot, -ch[t].nll.c);
        for (int a = 0; a < np; ++a) {
            kahan_add(&g[a], ch[t].g[a].s);
            kahan_add(&g[a], -ch[t].g[a].c);
            for (int b = a; b < np; ++b) {
                int k = a * np + b;
                kahan_add(&h[k], ch[t].h[k].s);
                kahan_add(&h[k], -ch[t].h[k].c);
                kahan_add(&hs[k], ch[t].hs[k].s);
                kahan_add(&hs[k], -ch[t].hs[k].c);
                kahan_add(&q[k], ch[t].w2[k].s);
                kahan_add(&q[k], -ch[t].w2[k].c);
            }
        }
        bad += ch[t].bad;
    }
    free(ch);
    if (bad) {
        *nll = INFINITY;
        return OR_ERR_NONPOSITIVE;
    }
    *nll = tot.s;
    for (int a = 0; a < np; ++a) {
        if (grad) grad[a] = g[a].s;
        for (int b = a; b < np; ++b) {
            int k = a * np + b;
            hess[a * np + b] = hess[b * np + a] = h[k].s;
            if (w2) w2[a * np + b] = w2[b * np + a] = q[k].s;
            if (hscale) hscale[a * np + b] = hscale[b * np + a] = hs[k].s;
        }
    }
    return OR_OK;
}

/* Per-event density P_i (for quadrature and special-case checks). */
int oracle_pdf(int kind, const double* ranges, const double* theta, const double* const* cols, int64_t n,
               double* out)
{
    model_t M;
    if (model_setup(&M, kind, ranges, theta) != OR_OK) return OR_ERR_ARG;
    int ndim = kind == OR_MASS1D ? 1 : 4;
    double x[4];
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < ndim; ++d) x[d] = cols[d][i];
        out[i] = event_density(&M, x, NULL);
    }
    return OR_OK;
}

/* Per-event gradient of ln P_i, row-major [n][npar] (for per-event checks). */
int oracle_dlogpdf(int kind, const double* ranges, const double* theta, const double* const* cols, int64_t n,
                   double* out)
{
    model_t M;
    if (model_setup(&M, kind, ranges, theta) != OR_OK) return OR_ERR_ARG;
    int ndim = kind == OR_MASS1D ? 1 : 4;
    double x[4], dP[OR_MAXPAR];
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < ndim; ++d) x[d] = cols[d][i];
        double P = event_density(&M, x, dP);
        for (int k = 0; k < M.npar; ++k) out[i * M.npar + k] = dP[k] / P;
    }
    return OR_OK;
}

/* The eleven Eq. 3 terms f_i(ctl, ctk, phi) per event, row-major [n][11]. */
void oracle_angular_terms(const double* ctl, const double* ctk, const double* phi, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) angular_terms(ctl[i], ctk[i], phi[i], out + 11 * i);
}

/* Normalisations: [N1, dlnN1/dmu, dlnN1/dsigma, N2, dlnN2/dalpha] for a mass window. */
void oracle_mass_norms(double ma, double mb, double mu, double sigma, double alpha, double* out)
{
    mass_norm_t n;
    mass_norm(&n, ma, mb, mu, sigma, alpha);
    out[0] = n.N1;
    out[1] = n.dlnN1_dmu;
    out[2] = n.dlnN1_dsig;
    out[3] = n.N2;
    out[4] = n.dlnN2_dal;
}

/* Second derivatives of the normalisations: [d2lnN1/dmu2, d2lnN1/dmu dsigma, d2lnN1/dsigma2,
 * d2lnN2/dalpha2]. */
void oracle_mass_norms2(double ma, double mb, double mu, double sigma, double alpha, double* out)
{
    mass_norm_t n;
    mass_norm(&n, ma, mb, mu, sigma, alpha);
    out[0] = n.d2lnN1[0];
    out[1] = n.d2lnN1[1];
    out[2] = n.d2lnN1[2];
    out[3] = n.d2lnN2_dal2;
}

/* Per-event second derivatives of ln P_i, row-major [n][npar][npar] (for per-event checks). */
int oracle_d2logpdf(int kind, const double* ranges, const double* theta, const double* const* cols, int64_t n,
                    double* out)
{
    model_t M;
    if (model_setup(&M, kind, ranges, theta) != OR_OK) return OR_ERR_ARG;
    int ndim = kind == OR_MASS1D ? 1 : 4;
    int np = M.npar;
    double x[4], dP[OR_MAXPAR], d2P[OR_MAXPAR * OR_MAXPAR];
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < ndim; ++d) x[d] = cols[d][i];
        double P = event_density(&M, x, dP);
        event_second(&M, x, d2P);
        for (int a = 0; a < np; ++a)
            for (int b = 0; b < np; ++b)
                out[(i * np + a) * np + b] = d2P[a * np + b] / P - (dP[a] / P) * (dP[b] / P);
    }
    return OR_OK;
}

int oracle_num_params(int kind) { return npar_of(kind); }
