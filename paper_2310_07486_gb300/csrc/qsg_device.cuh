// qsg_device.cuh -- device-side building blocks shared by the sm_103a kernels:
// the group descriptor, Philox4x32-10 and the bitsliced arithmetic on
// multispin words (bit b of a word = disorder sample b, set bit = spin -1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qsg {

enum : uint32_t { STREAM_J = 1u, STREAM_INIT = 2u, STREAM_SWEEP = 3u, STREAM_PT = 4u };

// Everything a kernel needs to know about one group of samples.  Plain data,
// copied by value into kernel arguments.
struct Group {
    int L, Ltau, W, R, K, algo, boundary, gid;
    int N;          // L * L * Ltau sites (= words per slot)
    int nslots;     // W * R * K
    int nlag;       // Ltau / 2 + 1
    int n_samples;
    int nwx;        // ceil(L * L / 64): words of one x-packed slice of one sample
    uint64_t *S;    // [nslots][Ltau][L][L]
    uint64_t *Jx;   // [W][L][L]  bond (x,y)-(x+1,y)
    uint64_t *Jy;   // [W][L][L]  bond (x,y)-(x,y+1)
    uint32_t *thr;  // [K][16]: [0..2] Metropolis S h = 2,4,6 ; [8..14] heat bath n_neg = 0..6
    uint64_t *ptA;  // concatenated A_i tables
    int32_t *ptA_off, *ptA_len;  // [K-1]
    uint64_t *ptB;  // [K-1][64]
    int32_t *U;     // [nslots][64] unsatisfied bonds of each slot and sample bit
    uint32_t *swapmask;  // [W*R][K-1][2] 32-bit halves of the per-pair swap masks
    unsigned long long *acc;  // [W*64][K-1] accepted swaps (summed over replicas)
    long long *Cacc, *Qacc;   // [R][W*64][K][nlag]
    long long *Pacc;          // [W*64][K]  sum of Q_ab^2 over slices and replica pairs
    unsigned long long *P4acc;  // [W*64][K][2] sum of Q_ab^4: low 32 bits and high bits summed apart
    long long *T3acc;         // [W*64][K] sum of Q_ab Q_bc Q_ca over slices and replica triples
    long long *Gacc, *F3acc;  // [W*64][K][L/2+1] momentum sums binned by x-distance
    long long *PPacc;         // [W*64][K][R(R-1)/2] sum of Q_ab^2 of each replica pair
    double *outC, *outQ, *outP;
    double *outO;             // [W*64][K][7] one-time observables of every sample
    double *outK;             // [K][8] disorder averages
    double *wcos;             // [L/2+1] cos(2 pi d / L), host FP64
    double xi_norm;           // 2 sin(pi / L), host FP64
    unsigned *arrivals;  // [nslots][L_tau/4] boundary arrival counters of the wavefront sweep
    int upb;             // work units per block of the generic wavefront kernel (0 = automatic)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t pick(const uint4 &v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// Bitsliced arithmetic.  count6 returns the 3-bit count (b2 b1 b0) of set bits
// among six words, bit position by bit position, with two full adders and a
// final 3-input add.  ge_scalar(b, m) is the word of positions whose count is
// >= the scalar m (0..7), an MSB-first comparison.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T maj3(T a, T b, T c) { return (a & b) | (c & (a ^ b)); }

template <typename T>
__device__ __forceinline__ void count6(T a, T b, T c, T d, T e, T f, T &b0, T &b1, T &b2) {
    const T s1 = a ^ b ^ c, c1 = maj3(a, b, c);
    const T s2 = d ^ e ^ f, c2 = maj3(d, e, f);
    b0 = s1 ^ s2;
    const T k = s1 & s2;
    b1 = c1 ^ c2 ^ k;
    b2 = maj3(c1, c2, k);
}

template <typename T>
__device__ __forceinline__ T ge_scalar(T b0, T b1, T b2, uint32_t m) {
    const T m0 = (m & 1u) ? ~T(0) : T(0);
    const T m1 = (m & 2u) ? ~T(0) : T(0);
    const T m2 = (m & 4u) ? ~T(0) : T(0);
    const T g0 = b0 | ~m0;
    const T g1 = (b1 & ~m1) | (~(b1 ^ m1) & g0);
    return (b2 & ~m2) | (~(b2 ^ m2) & g1);
}

// Number of table entries strictly above u; the tables are non-increasing in
// their index, so "u < T[n]" holds exactly for n < this count.
__device__ __forceinline__ uint32_t count_above3(uint32_t u, const uint32_t *t) {
    return (uint32_t)(u < t[0]) + (uint32_t)(u < t[1]) + (uint32_t)(u < t[2]);
}
__device__ __forceinline__ uint32_t count_above7(uint32_t u, const uint32_t *t) {
    uint32_t a = 0;
#pragma unroll
    for (int n = 0; n < 7; ++n) a += (uint32_t)(u < t[n]);
    return a;
}

}  // namespace qsg
