// judge.cpp -- the log-binning thermalisation check that judges a run (plain
// or learned ladder): host FP64, a component of this library (the paper
// instead tests the tempering dynamics).
//
// Bins of sweeps [2^m, 2^(m+1)).  For every sample, the bin mean of the
// energy per site of each replica and of q^2 of each replica pair, averaged
// over the ladder's k values; their mean over replicas (pairs) and its
// standard error.  A sample is thermalised at the first bin m >= n_last - 1
// that agrees with each of the n_last - 1 bins before it within one combined
// standard error sqrt(se_m^2 + se_i^2), for both observables.
#include <cmath>
#include <vector>

#include "qsg.h"

namespace {

// k-averaged value of replica (pair) r: a[r * rs + k * ks], k < K
double kavg(const double *a, int K, size_t ks) {
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += a[(size_t)k * ks];
    return s / K;
}

void mean_se(const double *v, int n, double *mean, double *se) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    const double m = s / n;
    double var = 0.0;
    for (int i = 0; i < n; ++i) var += (v[i] - m) * (v[i] - m);
    *mean = m;
    *se = std::sqrt(var / ((double)n * (n - 1)));
}

}  // namespace

extern "C" qsg_status qsg_judge(const double *E_bins, const double *q_bins, int32_t n_bins, int32_t n_samples,
                                int32_t n_replicas, int32_t n_k, int32_t n_pairs, int32_t n_last,
                                int32_t *first_pass) {
    if (!E_bins || !q_bins || !first_pass || n_bins < 0 || n_samples < 0 || n_replicas < 2 || n_k < 1 ||
        n_pairs < 2 || n_last < 2)
        return QSG_ERR_ARG;
    const int R = n_replicas, K = n_k, P = n_pairs;
    // per bin and sample: mean and standard error of the k-averaged E (over
    // replicas) and q^2 (over pairs)
    std::vector<double> Em((size_t)n_bins * n_samples), Es(Em.size()), qm(Em.size()), qs(Em.size());
    std::vector<double> tmp(R > P ? R : P);
    for (int m = 0; m < n_bins; ++m)
        for (int b = 0; b < n_samples; ++b) {
            const size_t c = (size_t)m * n_samples + b;
            for (int r = 0; r < R; ++r) tmp[r] = kavg(E_bins + (c * R + r) * K, K, 1);
            mean_se(tmp.data(), R, &Em[c], &Es[c]);
            for (int p = 0; p < P; ++p) tmp[p] = kavg(q_bins + c * K * P + p, K, (size_t)P);
            mean_se(tmp.data(), P, &qm[c], &qs[c]);
        }
    for (int b = 0; b < n_samples; ++b) {
        first_pass[b] = -1;
        for (int m = n_last - 1; m < n_bins && first_pass[b] < 0; ++m) {
            bool ok = true;
            const size_t c = (size_t)m * n_samples + b;
            for (int i = 1; i < n_last; ++i) {
                const size_t d = (size_t)(m - i) * n_samples + b;
                if (std::fabs(Em[c] - Em[d]) > std::sqrt(Es[c] * Es[c] + Es[d] * Es[d])) ok = false;
                if (std::fabs(qm[c] - qm[d]) > std::sqrt(qs[c] * qs[c] + qs[d] * qs[d])) ok = false;
            }
            if (ok) first_pass[b] = m;
        }
    }
    return QSG_OK;
}
