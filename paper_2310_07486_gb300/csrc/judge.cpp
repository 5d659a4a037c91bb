// judge.cpp -- the log-binning thermalisation check that judges a run (plain
// or learned ladder): host FP64, a component of this library (the paper
// instead tests the tempering dynamics).
//
// Bins of sweeps [2^m, 2^(m+1)).  For every sample, the bin mean of the
// energy per site of each replica and of q^2 of each replica pair, averaged
// over the ladder's k values.  Energy: mean over replicas, standard error
// from their spread.  q^2: mean over pairs, standard error by the jackknife
// over replicas (leaving out replica r drops the pairs that contain it; pairs
// sharing a replica are not independent).  A sample is thermalised at the
// first bin m >= n_last - 1 that agrees with each of the n_last - 1 bins
// before it within n_sigma combined standard errors, for both observables.
#include <cmath>
#include <vector>

#include "qsg.h"

namespace {

double kavg(const double *a, int K, size_t ks) {
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += a[(size_t)k * ks];
    return s / K;
}

}  // namespace

extern "C" qsg_status qsg_judge(const double *E_bins, const double *q_bins, int32_t n_bins, int32_t n_samples,
                                int32_t n_replicas, int32_t n_k, int32_t n_last, double n_sigma,
                                int32_t *first_pass) {
    if (!E_bins || !q_bins || !first_pass || n_bins < 0 || n_samples < 0 || n_replicas < 3 || n_k < 1 ||
        n_last < 2 || !(n_sigma > 0.0))
        return QSG_ERR_ARG;
    const int R = n_replicas, K = n_k, P = R * (R - 1) / 2;
    std::vector<int> pa(P), pb(P);
    for (int a = 0, i = 0; a < R; ++a)
        for (int b = a + 1; b < R; ++b, ++i) {
            pa[i] = a;
            pb[i] = b;
        }
    std::vector<double> Em((size_t)n_bins * n_samples), Es(Em.size()), qm(Em.size()), qs(Em.size());
    std::vector<double> e(R), q(P), jk(R);
    for (int m = 0; m < n_bins; ++m)
        for (int b = 0; b < n_samples; ++b) {
            const size_t c = (size_t)m * n_samples + b;
            double s = 0.0;
            for (int r = 0; r < R; ++r) {
                e[r] = kavg(E_bins + (c * R + r) * K, K, 1);
                s += e[r];
            }
            const double mean = s / R;
            double v = 0.0;
            for (int r = 0; r < R; ++r) v += (e[r] - mean) * (e[r] - mean);
            Em[c] = mean;
            Es[c] = std::sqrt(v / ((double)R * (R - 1)));
            double qsum = 0.0;
            for (int p = 0; p < P; ++p) {
                q[p] = kavg(q_bins + c * K * P + p, K, (size_t)P);
                qsum += q[p];
            }
            qm[c] = qsum / P;
            double jsum = 0.0;
            for (int r = 0; r < R; ++r) {
                double t = 0.0;
                int n = 0;
                for (int p = 0; p < P; ++p)
                    if (pa[p] != r && pb[p] != r) {
                        t += q[p];
                        ++n;
                    }
                jk[r] = t / n;
                jsum += jk[r];
            }
            const double jm = jsum / R;
            double jv = 0.0;
            for (int r = 0; r < R; ++r) jv += (jk[r] - jm) * (jk[r] - jm);
            qs[c] = std::sqrt((double)(R - 1) / R * jv);
        }
    for (int b = 0; b < n_samples; ++b) {
        first_pass[b] = -1;
        for (int m = n_last - 1; m < n_bins && first_pass[b] < 0; ++m) {
            bool ok = true;
            const size_t c = (size_t)m * n_samples + b;
            for (int i = 1; i < n_last; ++i) {
                const size_t d = (size_t)(m - i) * n_samples + b;
                if (std::fabs(Em[c] - Em[d]) > n_sigma * std::sqrt(Es[c] * Es[c] + Es[d] * Es[d])) ok = false;
                if (std::fabs(qm[c] - qm[d]) > n_sigma * std::sqrt(qs[c] * qs[c] + qs[d] * qs[d])) ok = false;
            }
            if (ok) first_pass[b] = m;
        }
    }
    return QSG_OK;
}
