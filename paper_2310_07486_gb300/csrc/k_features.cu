// k_features.cu -- the 64 per-sample coupling features of the learned k-ladder
// predictor (a component of this library, not of the paper; the definitions
// are listed with qsg_sample_features in qsg.h).
//
// The coupling bit-planes hold 64 samples per word, so the frustration of a
// plaquette is one XOR of four words for 64 samples at once: a plaquette is
// frustrated when an odd number of its bonds are negative.  One block per word
// of samples, one thread per sample bit; every thread reads the same words
// (broadcast) and counts its own bit.
#include "qsg_launch.h"

namespace qsg {

__global__ void __launch_bounds__(64) k_features(Group g, float *__restrict__ out) {
    const int w = blockIdx.x, b = threadIdx.x;
    const int L = g.L, n = L * L;
    const uint64_t *Jx = g.Jx + (size_t)w * n, *Jy = g.Jy + (size_t)w * n;
    auto jx = [&](int x, int y) { return (int)((Jx[y * L + x] >> b) & 1ull); };
    auto jy = [&](int x, int y) { return (int)((Jy[y * L + x] >> b) & 1ull); };
    // frustrated plaquette with lower-left corner (x, y)
    auto fr = [&](int x, int y) {
        x = (x % L + L) % L;
        y = (y % L + L) % L;
        const int x1 = x + 1 == L ? 0 : x + 1, y1 = y + 1 == L ? 0 : y + 1;
        return jx(x, y) ^ jy(x1, y) ^ jx(x, y1) ^ jy(x, y);
    };
    int cnt[64];
    for (int i = 0; i < 64; ++i) cnt[i] = 0;
    int cell_tot[16];
    for (int i = 0; i < 16; ++i) cell_tot[i] = 0;
    int nblocks = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const int F = fr(x, y);
            cnt[0] += F;
            const int xm = x == 0 ? L - 1 : x - 1, ym = y == 0 ? L - 1 : y - 1;
            const int nneg = jx(x, y) + jx(xm, y) + jy(x, y) + jy(x, ym);
            cnt[5 - nneg] += 1;  // bond sum 4 - 2 nneg -> bins -4, -2, 0, 2, 4 = 1..5
            cnt[6 + F + fr(xm, y) + fr(x, ym) + fr(xm, ym)] += 1;
            if ((x & 1) == 0 && (y & 1) == 0 && x + 1 < L && y + 1 < L) {
                cnt[11 + F + fr(x + 1, y) + fr(x, y + 1) + fr(x + 1, y + 1)] += 1;
                ++nblocks;
            }
            const int c = (4 * y / L) * 4 + (4 * x / L);
            cnt[16 + c] += F;
            cell_tot[c] += 1;
            cnt[32] += F & fr(x + 1, y + 1);
            cnt[33] += F & fr(x + 1, y - 1);
            cnt[34] += jx(x, y);
            cnt[35] += jy(x, y);
            for (int d = 1; d <= 8; ++d) {
                cnt[47 + d] += F & fr(x + d, y);
                cnt[55 + d] += F & fr(x, y + d);
            }
        }
    for (int y = 0; y < L; ++y) {
        int r = 0;
        for (int x = 0; x < L; ++x) r += fr(x, y);
        const int bin = 6 * r / L;
        cnt[36 + (bin > 5 ? 5 : bin)] += 1;
    }
    for (int x = 0; x < L; ++x) {
        int r = 0;
        for (int y = 0; y < L; ++y) r += fr(x, y);
        const int bin = 6 * r / L;
        cnt[42 + (bin > 5 ? 5 : bin)] += 1;
    }
    // each count over its number of cases, in FP64, rounded once to FP32
    float *o = out + ((size_t)w * 64 + b) * 64;
    const double dn = (double)n;
    for (int i = 0; i < 64; ++i) {
        double den = dn;
        if (i >= 11 && i <= 15) den = (double)nblocks;
        if (i >= 16 && i <= 31) den = (double)cell_tot[i - 16];
        if (i >= 36 && i <= 47) den = (double)L;
        o[i] = den > 0.0 ? (float)__ddiv_rn((double)cnt[i], den) : 0.0f;
    }
}

cudaError_t launch_features(const Group &g, float *out, cudaStream_t st) {
    count_launches(1);
    k_features<<<g.W, 64, 0, st>>>(g, out);
    return cudaGetLastError();
}

}  // namespace qsg
