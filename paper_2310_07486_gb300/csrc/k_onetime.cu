// k_onetime.cu -- one-time observables (Methods, "One-time observables";
// Eqs. (def-M), (chi-r), (xi-r), (Binder)) and the linear susceptibility
// (Sect. "On the magnetic susceptibilities").
//
// M_xy = <S_x S_y> at equal imaginary time is estimated with independent
// replicas a, b, c of one sample at one k, at every slice tau:
//   Tr M^2       <- Q_ab^2          Q_ab = sum_x S^a_x S^b_x
//   sum <SSSS>^2 <- Q_ab^4
//   Tr M^3       <- Q_ab Q_bc Q_ca
//   Tr Mhat M    <- |Q_ab(p)|^2     Q(p) = sum_x S^a_x S^b_x e^{i p.x}
//   Tr Mhat M^2  <- Re Q_su(p) Q_sv(-p) Q_uv   (s = each of a, b, c)
// for p = (2 pi / L, 0) and (0, 2 pi / L).  With n_c the overlap summed over
// the sites of column (row) c, |Q(p)|^2 = sum_d cos(2 pi d / L) G[d] where
// G[d] = sum_c n_c n_{c+d}; the kernel accumulates the integer sums G[d]
// (folded d ~ L - d) and the finish applies the cosines, so the accumulation
// is exact.  With a_c the number of sites of column c where the two replicas
// differ (n_c = L - 2 a_c) and A = sum_c a_c,
//   sum_c n_c n_{c+d} = L^3 - 4 L A + 4 sum_c a_c a_{c+d},
// and the last sum is a dot product of byte vectors (four columns per
// __dp4a); the column counts come from a bitsliced vertical add of the L row
// words of the slice.
//
// Input: the transposed scratch of the correlator pass ([pair][r][bit][tau]
// [nwx] x-packed slices, bit n = y L + x of word n / 64).  One block per
// (ladder pair of the batch, sample bit), one thread per slice.
#include <type_traits>

#include "qsg_launch.h"

namespace qsg {

constexpr int kMaxTripleR = 8;  // three-replica terms for 3 <= R <= 8
// Replica pairs whose Q^2 sums a block keeps in shared memory; with more
// (R > 128) every slice adds its pair sums straight to the global ones.
constexpr int kMaxSharedPairs = 8192;

__host__ __device__ constexpr int bit_length(int n) { return n == 0 ? 0 : 1 + bit_length(n >> 1); }

// Sizes for lattice side L: NW words per slice, NP packed byte words per
// count vector (4 columns per word, zero beyond L), NPL bit planes of a count
// (<= L), ND words of the doubled cyclic copy read by the shifted windows.
template <int L>
struct OtSize {
    static constexpr int NW = (L * L + 63) / 64;
    static constexpr int NP = (L + 3) / 4;
    static constexpr int NPL = bit_length(L);
    static constexpr int ND = ((L - 1) + 4 * (NP - 1)) / 4 + 2;
};

// Pack four small non-negative ints into bytes 0..3.
__device__ __forceinline__ uint32_t pack_bytes(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
    return __byte_perm(__byte_perm(b0, b1, 0x0040), __byte_perm(b2, b3, 0x0040), 0x5410);
}

// Difference counts of one replica pair at one slice: ca (columns) and cb
// (rows) as byte vectors [NP] (byte k of word w = count of column / row
// 4 w + k), and the total A = number of sites where the replicas differ.
template <int L>
__device__ __forceinline__ void diff_counts(const uint64_t *__restrict__ X, const uint64_t *__restrict__ Y,
                                            uint32_t (&ca)[OtSize<L>::NP], uint32_t (&cb)[OtSize<L>::NP], int &A) {
    constexpr int NW = OtSize<L>::NW, NP = OtSize<L>::NP, NPL = OtSize<L>::NPL;
    uint64_t o[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) o[q] = X[q] ^ Y[q];
    // rows (bits r L .. r L + L - 1), their counts, and the vertical bitsliced
    // sum of the rows: bit c of plane j is bit j of column c's count; after
    // row r a count is at most r + 1, which bounds the carry chain
    uint32_t P[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) P[j] = 0u;
    uint32_t rb[4 * NP];
    A = 0;
#pragma unroll
    for (int r = 0; r < L; ++r) {
        constexpr uint64_t mask = (L == 64) ? ~0ull : ((1ull << L) - 1);
        const int off = r * L, q = off >> 6, sh = off & 63;
        uint64_t f = o[q] >> sh;
        if (sh + L > 64) f |= o[q + 1] << (64 - sh);
        const uint32_t row = (uint32_t)(f & mask);
        rb[r] = (uint32_t)__popc(row);
        A += (int)rb[r];
        uint32_t carry = row;
#pragma unroll
        for (int j = 0; j < NPL; ++j)
            if (j < bit_length(r + 1)) {
                const uint32_t t = P[j] & carry;
                P[j] ^= carry;
                carry = t;
            }
    }
#pragma unroll
    for (int r = L; r < 4 * NP; ++r) rb[r] = 0u;
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        cb[w] = pack_bytes(rb[4 * w], rb[4 * w + 1], rb[4 * w + 2], rb[4 * w + 3]);
        // bits 4w .. 4w+3 of every plane spread to the low bit of bytes 0..3
        uint32_t v = 0u;
#pragma unroll
        for (int j = 0; j < NPL; ++j) v |= (((P[j] >> (4 * w)) & 0xFu) * 0x00204081u & 0x01010101u) << j;
        ca[w] = v;
    }
}

// The doubled cyclic copy dd[b] = x[b mod L] of a byte vector x[NP] (bytes
// beyond L of x are 0); every word takes its four bytes from at most two
// words of x, chosen at compile time.
template <int L>
__device__ __forceinline__ void cyclic_copy(const uint32_t (&x)[OtSize<L>::NP], uint32_t (&dd)[OtSize<L>::ND]) {
#pragma unroll
    for (int k = 0; k < OtSize<L>::ND; ++k) {
        const int c0 = (4 * k) % L;
        const int wa = c0 / 4;
        int wb = wa;
        uint32_t sel = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = (4 * k + i) % L, w = c / 4;
            if (w != wa) wb = w;
            sel |= (uint32_t)((w == wa ? 0 : 4) + c % 4) << (4 * i);
        }
        dd[k] = __byte_perm(x[wa], x[wb], sel);
    }
}

// sum_c x[c] y[(c + o) mod L] for byte vectors x (zero beyond L) and the
// cyclic copy dd of y; o a compile-time offset.
template <int L, int O>
__device__ __forceinline__ int cyc_dot(const uint32_t (&x)[OtSize<L>::NP], const uint32_t (&dd)[OtSize<L>::ND]) {
    unsigned acc = 0u;
#pragma unroll
    for (int w = 0; w < OtSize<L>::NP; ++w) {
        constexpr int sh = O & 3;
        const int k = (O >> 2) + w;
        const uint32_t y = sh == 0 ? dd[k] : __byte_perm(dd[k], dd[k + 1], 0x3210u + 0x1111u * sh);
        acc = __dp4a(x[w], y, acc);
    }
    return (int)acc;
}

// Compile-time loop over d = 0 .. H with the body f(integral_constant<d>).
template <int D, int H, class F>
__device__ __forceinline__ void for_d(F &&f) {
    if constexpr (D <= H) {
        f(std::integral_constant<int, D>{});
        for_d<D + 1, H>(f);
    }
}

template <int L>
__global__ void __launch_bounds__(128, 3) k_onetime(Group g, int p0, const uint64_t *__restrict__ P, int triples) {
    constexpr int NW = OtSize<L>::NW, NP = OtSize<L>::NP, ND = OtSize<L>::ND, H = L / 2;
    constexpr int L3 = L * L * L;
    extern __shared__ __align__(16) unsigned char ot_smem[];
    const int R = g.R, Lt = g.Ltau, bd = blockDim.x, tid = threadIdx.x;
    const int npair = R * (R - 1) / 2;
    const bool do3 = triples && R >= 3 && R <= kMaxTripleR;
    const bool pp_shared = npair <= kMaxSharedPairs;
    const int npsh = pp_shared ? npair : 0;
    // [pair] per-pair sums of Q^2 (up to kMaxSharedPairs pairs); [2][L/2+1]
    // [thread] the thread's G and F3 sums (kept in shared memory to spare
    // registers); then (triples only) [pair][dir][word][thread] packed
    // column/row difference counts and [pair][thread] overlaps
    unsigned long long *ppsh = reinterpret_cast<unsigned long long *>(ot_smem);
    long long *accsh = reinterpret_cast<long long *>(ot_smem + (size_t)npsh * 8);
    const size_t o_n = (size_t)npsh * 8 + (size_t)2 * (H + 1) * bd * 8;
    uint32_t *nsh = reinterpret_cast<uint32_t *>(ot_smem + o_n);
    int16_t *qsh = reinterpret_cast<int16_t *>(ot_smem + o_n + (size_t)npair * 2 * NP * 4 * bd);
    for (int i = tid; i < npsh; i += bd) ppsh[i] = 0ull;
#pragma unroll
    for (int d = 0; d <= H; ++d) {
        accsh[(size_t)d * bd + tid] = 0;
        accsh[(size_t)(H + 1 + d) * bd + tid] = 0;
    }
    __syncthreads();
    const int pb = blockIdx.x / 64, b = blockIdx.x % 64;
    const int p = p0 + pb, w = p / g.K, j = p % g.K;
    unsigned long long *ppg =
        reinterpret_cast<unsigned long long *>(g.PPacc) + ((size_t)(w * 64 + b) * g.K + j) * npair;
    const size_t plane = (size_t)Lt * NW;
    const uint64_t *base = P + (size_t)pb * R * 64 * plane + (size_t)b * plane;

    long long p2 = 0, t3 = 0;
    unsigned long long p4lo = 0, p4hi = 0;
    for (int t = tid; t < Lt; t += bd) {
        int pi = 0;
        for (int ra = 0; ra < R; ++ra)
            for (int rb = ra + 1; rb < R; ++rb, ++pi) {
                uint32_t ca[NP], cb[NP];
                int A;
                diff_counts<L>(base + (size_t)ra * 64 * plane + (size_t)t * NW,
                               base + (size_t)rb * 64 * plane + (size_t)t * NW, ca, cb, A);
                const int q0 = L * L - 2 * A;
                const unsigned long long q2 = (unsigned long long)(q0 * q0);
                p2 += (long long)q2;
                atomicAdd(pp_shared ? &ppsh[pi] : &ppg[pi], q2);
                const unsigned long long q4 = q2 * q2;
                p4lo += q4 & 0xFFFFFFFFull;
                p4hi += q4 >> 32;
                // G[d] = sum_c nx_c nx_{c+d} + ny_c ny_{c+d}
                //      = 2 L^3 - 8 L A + 4 (sum_c a_c a_{c+d} + sum_r b_r b_{r+d})
                {
                    uint32_t dda[ND], ddb[ND];
                    cyclic_copy<L>(ca, dda);
                    cyclic_copy<L>(cb, ddb);
                    for_d<0, H>([&](auto dc) {
                        constexpr int d = decltype(dc)::value;
                        const int sv = 2 * L3 - 8 * L * A + 4 * (cyc_dot<L, d>(ca, dda) + cyc_dot<L, d>(cb, ddb));
                        accsh[(size_t)d * bd + tid] += (d == 0 || d == H) ? sv : 2 * sv;  // G[d] = G[L - d]
                    });
                }
                if (do3) {
#pragma unroll
                    for (int w = 0; w < NP; ++w) {
                        nsh[(((size_t)pi * 2 + 0) * NP + w) * bd + tid] = ca[w];
                        nsh[(((size_t)pi * 2 + 1) * NP + w) * bd + tid] = cb[w];
                    }
                    qsh[(size_t)pi * bd + tid] = (int16_t)q0;
                }
            }
        if (!do3) continue;
        // pair index of (a, b), a < b: a (2R - a - 1) / 2 + (b - a - 1)
        auto pid = [R](int a, int b2) { return a * (2 * R - a - 1) / 2 + (b2 - a - 1); };
        for (int ra = 0; ra < R; ++ra)
            for (int rb = ra + 1; rb < R; ++rb)
                for (int rc = rb + 1; rc < R; ++rc) {
                    const int ab = pid(ra, rb), bc = pid(rb, rc), ac = pid(ra, rc);
                    const long long qab = qsh[(size_t)ab * bd + tid], qbc = qsh[(size_t)bc * bd + tid],
                                    qac = qsh[(size_t)ac * bd + tid];
                    t3 += qab * qbc * qac;
                    int ft[H + 1];  // this triple's F3 sums (int32: < 6 * 2^10 * 2^16)
#pragma unroll
                    for (int d = 0; d <= H; ++d) ft[d] = 0;
                    // the replica shared by the two momentum-carrying overlaps: a, b, c
#pragma unroll 1
                    for (int rot = 0; rot < 3; ++rot) {
                        const int p1 = rot == 0 ? ab : (rot == 1 ? ab : ac);
                        const int p2i = rot == 0 ? ac : bc;
                        const long long qz = rot == 0 ? qbc : (rot == 1 ? qac : qab);
                        // difference totals of the two pairs: A = (L^2 - q) / 2
                        const int A1 = (L * L - (int)(p1 == ab ? qab : qac)) / 2;
                        const int A2 = (L * L - (int)(p2i == ac ? qac : qbc)) / 2;
#pragma unroll
                        for (int dir = 0; dir < 2; ++dir) {
                            uint32_t a1[NP], a2[NP], dd2[ND];
#pragma unroll
                            for (int w = 0; w < NP; ++w) {
                                a1[w] = nsh[(((size_t)p1 * 2 + dir) * NP + w) * bd + tid];
                                a2[w] = nsh[(((size_t)p2i * 2 + dir) * NP + w) * bd + tid];
                            }
                            cyclic_copy<L>(a2, dd2);
                            // sum_c n1_c (n2_{c+d} + n2_{c-d}) with n = L - 2 a (one term at d = 0, L/2)
                            for_d<0, H>([&](auto dc) {
                                constexpr int d = decltype(dc)::value;
                                int sv;
                                if (d == 0 || d == H)
                                    sv = L3 - 2 * L * (A1 + A2) + 4 * cyc_dot<L, d>(a1, dd2);
                                else
                                    sv = 2 * L3 - 4 * L * (A1 + A2) +
                                         4 * (cyc_dot<L, d>(a1, dd2) + cyc_dot<L, (L - d) % L>(a1, dd2));
                                ft[d] += (int)qz * sv;
                            });
                        }
                    }
#pragma unroll
                    for (int d = 0; d <= H; ++d) accsh[(size_t)(H + 1 + d) * bd + tid] += ft[d];
                }
    }

    __syncthreads();
    for (int i = tid; i < npsh; i += bd) atomicAdd(&ppg[i], ppsh[i]);
    // block reduction: warp shuffles, one atomic per warp and quantity
    auto wsum = [](long long v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        return v;
    };
    const size_t idx = (size_t)(w * 64 + b) * g.K + j;
    const bool lead = (tid & 31) == 0;
    {
        const long long a = wsum(p2), c3 = wsum(t3);
        const long long lo = wsum((long long)p4lo), hi = wsum((long long)p4hi);
        if (lead) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&g.Pacc[idx]), (unsigned long long)a);
            atomicAdd(&g.P4acc[2 * idx], (unsigned long long)lo);
            atomicAdd(&g.P4acc[2 * idx + 1], (unsigned long long)hi);
            if (do3) atomicAdd(reinterpret_cast<unsigned long long *>(&g.T3acc[idx]), (unsigned long long)c3);
        }
    }
#pragma unroll
    for (int d = 0; d <= H; ++d) {
        const long long gs = wsum(accsh[(size_t)d * bd + tid]);
        const long long fs = wsum(accsh[(size_t)(H + 1 + d) * bd + tid]);
        if (lead) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&g.Gacc[idx * (H + 1) + d]), (unsigned long long)gs);
            if (do3)
                atomicAdd(reinterpret_cast<unsigned long long *>(&g.F3acc[idx * (H + 1) + d]),
                          (unsigned long long)fs);
        }
    }
}

size_t onetime_smem_bytes(const Group &g, int triples, int threads) {
    const int npair = g.R * (g.R - 1) / 2;
    const size_t pp = (size_t)(npair <= kMaxSharedPairs ? npair : 0) * 8 + (size_t)2 * (g.L / 2 + 1) * threads * 8;
    if (!triples || g.R < 3 || g.R > kMaxTripleR) return pp;
    const int np4 = 4 * ((g.L + 3) / 4);  // packed count bytes per vector
    return pp + (size_t)npair * (2 * np4 + 2) * threads;
}

template <int L>
static cudaError_t launch_onetime_L(const Group &g, int p0, int np, const uint64_t *P, int triples,
                                    cudaStream_t st) {
    int threads = 128;
    while (threads > 32 && onetime_smem_bytes(g, triples, threads) > 96 * 1024) threads /= 2;
    const size_t sm = onetime_smem_bytes(g, triples, threads);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_onetime<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    count_launches(1);
    k_onetime<L><<<np * 64, threads, sm, st>>>(g, p0, P, triples);
    return cudaGetLastError();
}

cudaError_t launch_onetime(const Group &g, int p0, int np, const uint64_t *P, int triples, cudaStream_t st) {
    if (g.R < 2) return cudaSuccess;
    switch (g.L) {
        case 2: return launch_onetime_L<2>(g, p0, np, P, triples, st);
        case 4: return launch_onetime_L<4>(g, p0, np, P, triples, st);
        case 6: return launch_onetime_L<6>(g, p0, np, P, triples, st);
        case 8: return launch_onetime_L<8>(g, p0, np, P, triples, st);
        case 10: return launch_onetime_L<10>(g, p0, np, P, triples, st);
        case 12: return launch_onetime_L<12>(g, p0, np, P, triples, st);
        case 14: return launch_onetime_L<14>(g, p0, np, P, triples, st);
        case 16: return launch_onetime_L<16>(g, p0, np, P, triples, st);
        case 18: return launch_onetime_L<18>(g, p0, np, P, triples, st);
        case 20: return launch_onetime_L<20>(g, p0, np, P, triples, st);
        case 22: return launch_onetime_L<22>(g, p0, np, P, triples, st);
        case 24: return launch_onetime_L<24>(g, p0, np, P, triples, st);
        case 26: return launch_onetime_L<26>(g, p0, np, P, triples, st);
        case 28: return launch_onetime_L<28>(g, p0, np, P, triples, st);
        case 30: return launch_onetime_L<30>(g, p0, np, P, triples, st);
        case 32: return launch_onetime_L<32>(g, p0, np, P, triples, st);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// FP64 finish.  Per (sample bit, k): q2, q4, chi2, F2, chi3, F3, chi_lin with
// the normalisations of Eqs. (chi-r), (Binder) (one IEEE division each) and
// chi_lin = C(0) + 2 sum_{0 < tau < L_tau/2} C(tau) + C(L_tau/2), C averaged
// over replicas.  Per k: disorder averages over the group's samples and
// xi = sqrt(chi / F - 1) / (2 sin(pi / L)), B = mean q4 / (mean q2)^2.
// ---------------------------------------------------------------------------
__global__ void k_onetime_finish(Group g, double nm, int triples) {
    const int H = g.L / 2, R = g.R, K = g.K, nl = g.nlag;
    const double LD = (double)(g.L * g.L), Lt = (double)g.Ltau;
    const double npair = (double)(R * (R - 1) / 2), ntrip = (double)(R * (R - 1) * (R - 2) / 6);
    const bool has3 = triples && R >= 3 && R <= kMaxTripleR;
    const int total = g.n_samples * K;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int s = i / K, j = i % K;
        const size_t c = (size_t)s * K + j;  // the sample index equals the bit index w * 64 + b
        double G = 0.0, F3 = 0.0;
        for (int d = 0; d <= H; ++d) {
            G = __dadd_rn(G, __dmul_rn(g.wcos[d], (double)g.Gacc[c * (H + 1) + d]));
            F3 = __dadd_rn(F3, __dmul_rn(g.wcos[d], (double)g.F3acc[c * (H + 1) + d]));
        }
        const double p4 = __dadd_rn(__dmul_rn((double)g.P4acc[2 * c + 1], 4294967296.0), (double)g.P4acc[2 * c]);
        double *o = g.outO + c * 7;
        o[0] = __ddiv_rn((double)g.Pacc[c], nm * npair * LD * LD * Lt);
        o[1] = __ddiv_rn(p4, nm * npair * LD * LD * LD * LD * Lt);
        o[2] = __ddiv_rn((double)g.Pacc[c], nm * npair * Lt * LD);
        o[3] = __ddiv_rn(G, 2.0 * nm * npair * Lt * LD);
        o[4] = has3 ? __ddiv_rn((double)g.T3acc[c], nm * ntrip * Lt * LD) : __longlong_as_double(0x7ff8000000000000LL);
        o[5] = has3 ? __ddiv_rn(F3, 6.0 * nm * ntrip * Lt * LD) : __longlong_as_double(0x7ff8000000000000LL);
        double cl = 0.0;
        for (int r = 0; r < R; ++r) {
            const long long *Cr = g.Cacc + (((size_t)r * g.W * 64 + s) * K + j) * nl;
            double sr = 0.0;
            for (int lag = 0; lag < nl; ++lag) {
                const double v = __ddiv_rn((double)Cr[lag], __dmul_rn(__dmul_rn(nm, LD), Lt));
                sr = __dadd_rn(sr, (lag == 0 || lag == nl - 1) ? v : __dmul_rn(2.0, v));
            }
            cl = __dadd_rn(cl, sr);
        }
        o[6] = __ddiv_rn(cl, (double)R);
    }
}

__global__ void k_onetime_average(Group g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.K) return;
    const int K = g.K, ns = g.n_samples;
    double m[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int s = 0; s < ns; ++s)
        for (int f = 0; f < 7; ++f) m[f] = __dadd_rn(m[f], g.outO[((size_t)s * K + j) * 7 + f]);
    for (int f = 0; f < 7; ++f) m[f] = __ddiv_rn(m[f], (double)ns);
    const double s2 = g.xi_norm;  // 2 sin(pi / L), host FP64
    double *o = g.outK + (size_t)j * 8;
    o[0] = m[2];
    o[1] = m[3];
    o[2] = __ddiv_rn(sqrt(__ddiv_rn(m[2], m[3]) - 1.0), s2);
    o[3] = m[4];
    o[4] = m[5];
    o[5] = __ddiv_rn(sqrt(__ddiv_rn(m[4], m[5]) - 1.0), s2);
    o[6] = __ddiv_rn(m[1], __dmul_rn(m[0], m[0]));
    o[7] = m[6];
}

cudaError_t launch_onetime_finish(const Group &g, long long n_meas, int triples, cudaStream_t st) {
    const int total = g.n_samples * g.K;
    int blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_launches(2);
    k_onetime_finish<<<blocks, 256, 0, st>>>(g, (double)n_meas, triples);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_onetime_average<<<(g.K + 127) / 128, 128, 0, st>>>(g);
    return cudaGetLastError();
}

}  // namespace qsg
