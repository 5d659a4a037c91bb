// fits.cpp -- per-sample correlation lengths from the replica correlators
// (Methods, "Fitting process and Euclidean correlation length estimation"),
// host FP64, and the tau-tilde variable of Sect. "On the magnetic
// susceptibilities".
//
// For one sample at one k, from C(tau) and Q2(tau) of its R replicas at lags
// 0 .. L_tau/2:
//   1. replica mean and its standard error;
//   2. a constant fitted to Q2 on [L_tau/4, L_tau/2] (the plateau), weights
//      1/sigma^2, acceptable iff chi2/dof <= 2;
//   3. window tau_w,f = first lag >= 1 with f <= 3.5 sigma_f, f = C or
//      Q2 - Q_pl (tau_w,Q2 = L_tau/2, plateau free, when the constant fit is
//      not acceptable; eta not estimated when C never reaches 3.5 sigma);
//   4. C = B [e^{-tau/eta} + z e^{-(L_tau-tau)/eta}] on [tau_min, tau_w,C],
//      tau_min from tau_w,C / 10 up until chi2/dof < 1; Q2 = Q_pl + one or two
//      exponentials on [tau_min, tau_w,Q2], tau_min from 1 up until
//      chi2/dof < 0.5; the smaller chi2/dof is kept, eta_e = its largest eta.
// Lags with sigma = 0 (tau = 0, where C = Q2 = 1 exactly) carry no weight.
// A decay length beyond L_tau cannot be estimated: the minimiser keeps every
// decay length in (0, 10 L_tau], and a fit ending above L_tau marks its
// correlator (or its one- or two-term model) as not estimated.
// The minimiser is Levenberg-Marquardt with analytic derivatives; the
// parameter errors are the square roots of the diagonal of (J^T W J)^-1.
#include <cmath>
#include <cstring>
#include <vector>

#include "qsg.h"

namespace {

constexpr double kPlateauChi2 = 2.0, kWindowSigmas = 3.5, kChi2C = 1.0, kChi2Q = 0.5;
constexpr int kMaxPar = 5;

// Model: value and derivatives with respect to the parameters at lag t.
struct Model {
    int np = 0;
    double eta_max = INFINITY;  // decay lengths stay in (0, eta_max]
    virtual void eval(const double *p, double t, double *f, double *df) const = 0;
    virtual bool valid(const double *p) const = 0;  // decay lengths positive
    virtual ~Model() = default;
};

// B [e^{-t/eta} + z e^{-(Lt - t)/eta}], p = (B, eta)
struct CModel : Model {
    double Lt, z;
    CModel(double Lt_, double z_) : Lt(Lt_), z(z_) {
        np = 2;
        eta_max = 10.0 * Lt_;
    }
    void eval(const double *p, double t, double *f, double *df) const override {
        const double e1 = std::exp(-t / p[1]), e2 = std::exp(-(Lt - t) / p[1]);
        *f = p[0] * (e1 + z * e2);
        df[0] = e1 + z * e2;
        df[1] = p[0] * (e1 * t + z * e2 * (Lt - t)) / (p[1] * p[1]);
    }
    bool valid(const double *p) const override { return p[1] > 0.0 && p[1] <= eta_max; }
};

// Q_pl + sum_i B_i e^{-t/eta_i}; p = ([Q_pl,] B_1, eta_1, [B_2, eta_2])
struct QModel : Model {
    int nexp;
    bool free_pl;
    double qpl;
    QModel(int nexp_, bool free_pl_, double qpl_, double eta_max_) : nexp(nexp_), free_pl(free_pl_), qpl(qpl_) {
        np = 2 * nexp + (free_pl ? 1 : 0);
        eta_max = eta_max_;
    }
    void eval(const double *p, double t, double *f, double *df) const override {
        int o = 0;
        double v = qpl;
        if (free_pl) {
            v = p[0];
            df[0] = 1.0;
            o = 1;
        }
        for (int i = 0; i < nexp; ++i) {
            const double B = p[o + 2 * i], eta = p[o + 2 * i + 1], e = std::exp(-t / eta);
            v += B * e;
            df[o + 2 * i] = e;
            df[o + 2 * i + 1] = B * e * t / (eta * eta);
        }
        *f = v;
    }
    bool valid(const double *p) const override {
        const int o = free_pl ? 1 : 0;
        for (int i = 0; i < nexp; ++i)
            if (!(p[o + 2 * i + 1] > 0.0 && p[o + 2 * i + 1] <= eta_max)) return false;
        return true;
    }
};

// Solve A x = b (n <= kMaxPar) by Gaussian elimination with partial pivoting.
bool solve(int n, double A[kMaxPar][kMaxPar], double *b) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (!(std::fabs(A[piv][c]) > 0.0)) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c][k], A[piv][k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double m = A[r][c] / A[c][c];
            for (int k = c; k < n; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double v = b[r];
        for (int k = r + 1; k < n; ++k) v -= A[r][k] * b[k];
        b[r] = v / A[r][r];
    }
    return true;
}

struct Data {
    std::vector<double> t, y, s;
};

double chi2_of(const Model &m, const Data &d, const double *p) {
    double c = 0.0, f, df[kMaxPar];
    for (size_t i = 0; i < d.t.size(); ++i) {
        m.eval(p, d.t[i], &f, df);
        const double r = (f - d.y[i]) / d.s[i];
        c += r * r;
    }
    return c;
}

// Levenberg-Marquardt from p (in place); returns chi2, fills err.
double levmar(const Model &m, const Data &d, double *p, double *err) {
    const int np = m.np;
    double chi2 = chi2_of(m, d, p), lambda = 1e-3;
    double A[kMaxPar][kMaxPar], g[kMaxPar];
    auto normal = [&](const double *q) {
        for (int a = 0; a < np; ++a) {
            g[a] = 0.0;
            for (int b = 0; b < np; ++b) A[a][b] = 0.0;
        }
        double f, df[kMaxPar];
        for (size_t i = 0; i < d.t.size(); ++i) {
            m.eval(q, d.t[i], &f, df);
            const double w = 1.0 / (d.s[i] * d.s[i]), r = f - d.y[i];
            for (int a = 0; a < np; ++a) {
                g[a] += w * df[a] * r;
                for (int b = 0; b < np; ++b) A[a][b] += w * df[a] * df[b];
            }
        }
    };
    normal(p);
    // up to three passes: a pass that ends on a tiny step or a flat chi2 after
    // the damping has grown large may stop short in a long curved valley (the
    // two-exponential fits); a restart with the damping reset either moves
    // on or confirms the end point
    for (int pass = 0; pass < 3; ++pass) {
    const double chi2_start = chi2;
    lambda = 1e-3;
    for (int it = 0; it < 2000 && lambda < 1e30; ++it) {
        double M[kMaxPar][kMaxPar], step[kMaxPar], trial[kMaxPar];
        for (int a = 0; a < np; ++a) {
            for (int b = 0; b < np; ++b) M[a][b] = A[a][b];
            M[a][a] += lambda * (A[a][a] > 0.0 ? A[a][a] : 1.0);
            step[a] = -g[a];
        }
        if (!solve(np, M, step)) {
            lambda *= 10.0;
            continue;
        }
        for (int a = 0; a < np; ++a) trial[a] = p[a] + step[a];
        const double c2 = m.valid(trial) ? chi2_of(m, d, trial) : INFINITY;
        if (!(c2 < chi2)) {
            lambda *= 10.0;
            continue;
        }
        bool small = true;
        for (int a = 0; a < np; ++a)
            if (std::fabs(step[a]) > 1e-14 * (std::fabs(p[a]) + 1e-14)) small = false;
        const bool flat = chi2 - c2 <= 1e-15 * chi2;
        std::memcpy(p, trial, sizeof(double) * np);
        chi2 = c2;
        lambda = std::fmax(lambda * 0.1, 1e-15);
        normal(p);
        if (small || flat) break;
    }
    if (!(chi2 < chi2_start * (1.0 - 1e-12))) break;
    }
    // errors: sqrt of the diagonal of (J^T W J)^-1, column by column
    for (int a = 0; a < np; ++a) {
        double M[kMaxPar][kMaxPar], e[kMaxPar];
        for (int r = 0; r < np; ++r) {
            for (int c = 0; c < np; ++c) M[r][c] = A[r][c];
            e[r] = r == a ? 1.0 : 0.0;
        }
        err[a] = solve(np, M, e) ? std::sqrt(std::fabs(e[a])) : NAN;
    }
    return chi2;
}

// Straight line through log y of the positive points: amplitude and decay
// length to start the minimiser.
void loglin_guess(const Data &d, double *B, double *eta) {
    double st = 0, sy = 0, stt = 0, sty = 0;
    int n = 0;
    double first_pos = NAN;
    for (size_t i = 0; i < d.t.size(); ++i)
        if (d.y[i] > 0.0) {
            const double ly = std::log(d.y[i]);
            st += d.t[i];
            sy += ly;
            stt += d.t[i] * d.t[i];
            sty += d.t[i] * ly;
            if (n == 0) first_pos = d.y[i];
            ++n;
        }
    if (n >= 2) {
        const double den = n * stt - st * st;
        const double slope = (n * sty - st * sy) / den, icpt = (sy - slope * st) / n;
        if (slope < 0.0) {
            *B = std::exp(icpt);
            *eta = -1.0 / slope;
            return;
        }
    }
    *B = n > 0 ? first_pos : 1.0;
    *eta = std::fmax(1.0, (d.t.back() - d.t.front()) / 2.0);
}

Data gather(const double *y, const double *s, int lo, int hi) {
    Data d;
    for (int t = lo; t <= hi; ++t)
        if (s[t] > 0.0) {
            d.t.push_back((double)t);
            d.y.push_back(y[t]);
            d.s.push_back(s[t]);
        }
    return d;
}

int window(const double *f, const double *s, int half) {
    for (int t = 1; t <= half; ++t)
        if (f[t] <= kWindowSigmas * s[t]) return t;
    return -1;
}

void fit_C(const double *C, const double *s, int Lt, double z, qsg_fit_result *o) {
    const int half = Lt / 2;
    const int tw = window(C, s, half);
    o->C_tau_w = tw < 0 ? half : tw;
    if (tw < 0) return;  // eta beyond L_tau: not estimated
    CModel m((double)Lt, z);
    for (int tmin = tw / 10 > 1 ? tw / 10 : 1;; ++tmin) {
        Data d = gather(C, s, tmin, tw);
        const int dof = (int)d.t.size() - 2;
        if (dof < 1) return;
        double p[2], e[2];
        loglin_guess(d, &p[0], &p[1]);
        p[1] = std::fmin(p[1], m.eta_max);
        const double c2 = levmar(m, d, p, e);
        if (c2 / dof < kChi2C) {
            if (p[1] > (double)Lt) return;  // eta beyond L_tau: not estimated
            o->C_ok = 1;
            o->C_tau_min = tmin;
            o->eta = p[1];
            o->eta_err = e[1];
            o->C_amp = p[0];
            o->C_chi2dof = c2 / dof;
            return;
        }
    }
}

struct QFit {
    bool ok = false;
    double chi2dof = 0, p[kMaxPar] = {}, e[kMaxPar] = {};
    int tmin = 0;
};

QFit fit_Q_terms(const double *Q, const double *s, int tw, int nexp, double qpl, bool free_pl, int Lt) {
    QFit r;
    QModel m(nexp, free_pl, qpl, 10.0 * Lt);
    for (int tmin = 1; tmin <= tw; ++tmin) {
        Data d = gather(Q, s, tmin, tw);
        const int dof = (int)d.t.size() - m.np;
        if (dof < 1) return r;
        const double base = free_pl ? d.y.back() : qpl;
        Data sh = d;
        for (double &v : sh.y) v -= base;
        double B0, eta0;
        loglin_guess(sh, &B0, &eta0);
        double p[kMaxPar], e[kMaxPar];
        int o = 0;
        if (free_pl) p[o++] = base;
        if (nexp == 1) {
            p[o] = B0;
            p[o + 1] = eta0;
        } else {
            p[o] = 0.5 * B0;
            p[o + 1] = 2.0 * eta0;
            p[o + 2] = 0.5 * B0;
            p[o + 3] = 0.5 * eta0;
        }
        for (int i = 0; i < nexp; ++i) p[o + 2 * i + 1] = std::fmin(p[o + 2 * i + 1], m.eta_max);
        const double c2 = levmar(m, d, p, e);
        if (c2 / dof < kChi2Q) {
            for (int i = 0; i < nexp; ++i)
                if (p[o + 2 * i + 1] > (double)Lt) return r;  // beyond L_tau: not estimated
            r.ok = true;
            r.chi2dof = c2 / dof;
            r.tmin = tmin;
            std::memcpy(r.p, p, sizeof(p));
            std::memcpy(r.e, e, sizeof(e));
            return r;
        }
    }
    return r;
}

void fit_Q(const double *Q, const double *s, int Lt, qsg_fit_result *o) {
    const int half = Lt / 2, lo = (Lt + 3) / 4;
    double sw = 0, swq = 0;
    for (int t = lo; t <= half; ++t)
        if (s[t] > 0.0) {
            const double w = 1.0 / (s[t] * s[t]);
            sw += w;
            swq += w * Q[t];
        }
    int n = 0;
    double chi2 = 0.0;
    const double qpl = swq / sw;
    for (int t = lo; t <= half; ++t)
        if (s[t] > 0.0) {
            const double r = (Q[t] - qpl) / s[t];
            chi2 += r * r;
            ++n;
        }
    o->Q_pl = qpl;
    o->Q_pl_err = 1.0 / std::sqrt(sw);
    o->plateau_chi2dof = n > 1 ? chi2 / (n - 1) : 0.0;
    o->plateau_ok = o->plateau_chi2dof <= kPlateauChi2 ? 1 : 0;
    int tw = half;
    if (o->plateau_ok) {
        std::vector<double> f(half + 1);
        for (int t = 0; t <= half; ++t) f[t] = Q[t] - qpl;
        const int w = window(f.data(), s, half);
        tw = w < 0 ? half : w;
    }
    o->Q_tau_w = tw;
    const bool free_pl = !o->plateau_ok;
    QFit best;
    int best_n = 0;
    for (int nexp = 1; nexp <= 2; ++nexp) {
        QFit r = fit_Q_terms(Q, s, tw, nexp, qpl, free_pl, Lt);
        if (r.ok && (!best.ok || r.chi2dof < best.chi2dof)) {
            best = r;
            best_n = nexp;
        }
    }
    if (!best.ok) return;
    const int off = free_pl ? 1 : 0;
    int imax = 0;
    if (best_n == 2 && best.p[off + 3] > best.p[off + 1]) imax = 1;
    o->Q_ok = 1;
    o->Q_n_exp = best_n;
    o->Q_tau_min = best.tmin;
    o->Q_chi2dof = best.chi2dof;
    o->eta_e = best.p[off + 2 * imax + 1];
    o->eta_e_err = best.e[off + 2 * imax + 1];
    o->eta_2 = best_n == 2 ? best.p[off + 2 * (1 - imax) + 1] : NAN;
    if (free_pl) {
        o->Q_pl = best.p[0];
        o->Q_pl_err = best.e[0];
    }
}

}  // namespace

extern "C" {

void qsg_tau_tilde(int32_t Ltau, double *out) {
    if (!out || Ltau < 2) return;
    const double pi = 3.14159265358979323846;
    for (int t = 0; t <= Ltau / 2; ++t) out[t] = Ltau / pi * std::sin(pi * t / Ltau);
}

qsg_status qsg_fit_correlators(const double *C, const double *Q2, int32_t n_replicas, int64_t n_series, int32_t Ltau,
                               int32_t boundary, qsg_fit_result *out) {
    if (!C || !Q2 || !out || n_replicas < 2 || n_series < 0 || Ltau < 4 || (Ltau & 1)) return QSG_ERR_ARG;
    if (boundary != QSG_PBC && boundary != QSG_APBC) return QSG_ERR_ARG;
    const int nl = Ltau / 2 + 1, R = n_replicas;
    const double z = boundary == QSG_APBC ? -1.0 : 1.0;
    std::vector<double> mc(nl), sc(nl), mq(nl), sq(nl);
    for (int64_t i = 0; i < n_series; ++i) {
        for (int t = 0; t < nl; ++t) {
            double a = 0, b = 0;
            for (int r = 0; r < R; ++r) {
                a += C[((size_t)r * n_series + i) * nl + t];
                b += Q2[((size_t)r * n_series + i) * nl + t];
            }
            a /= R;
            b /= R;
            double va = 0, vb = 0;
            for (int r = 0; r < R; ++r) {
                const double da = C[((size_t)r * n_series + i) * nl + t] - a;
                const double db = Q2[((size_t)r * n_series + i) * nl + t] - b;
                va += da * da;
                vb += db * db;
            }
            mc[t] = a;
            mq[t] = b;
            sc[t] = std::sqrt(va / ((double)R * (R - 1)));
            sq[t] = std::sqrt(vb / ((double)R * (R - 1)));
        }
        qsg_fit_result *o = out + i;
        std::memset(o, 0, sizeof(*o));
        o->eta = o->eta_err = o->C_amp = o->C_chi2dof = NAN;
        o->eta_e = o->eta_e_err = o->eta_2 = o->Q_chi2dof = NAN;
        fit_C(mc.data(), sc.data(), Ltau, z, o);
        fit_Q(mq.data(), sq.data(), Ltau, o);
    }
    return QSG_OK;
}

}  // extern "C"
