// k_energy_pt.cu -- integer action of every configuration and the
// parallel-tempering step over the k ladder (Methods, "Simulation details").
#include "qsg_launch.h"

namespace qsg {

constexpr int kEnergyPlanes = 16;              // bits of a warp's count per sample (32 x 6 x kEnergyRun < 2^15)
constexpr int kEnergyRun = 128;                // tau planes per block (a multiple of 4)
constexpr int kEnergyBuf = 16;                 // planes in the shared-memory ring
constexpr int kEnergyAhead = kEnergyBuf - 5;   // planes in flight beyond the five being read
constexpr int kEnergyThirtyTwos = 5;           // planes of a thread's count of 32s (6 x kEnergyRun / 32 < 2^5)

// a += b for two bitsliced counters of kEnergyPlanes planes (ripple carry)
__device__ __forceinline__ void vadd_counter(uint64_t (&a)[kEnergyPlanes], const uint64_t (&b)[kEnergyPlanes]) {
    uint64_t carry = 0;
#pragma unroll
    for (int p = 0; p < kEnergyPlanes; ++p) {
        const uint64_t s = a[p] ^ b[p] ^ carry;
        carry = (a[p] & b[p]) | (carry & (a[p] ^ b[p]));
        a[p] = s;
    }
}

// carry-save adder: l = a ^ b ^ c (same weight), h = majority (twice the weight)
__device__ __forceinline__ void csa(uint64_t &h, uint64_t &l, uint64_t a, uint64_t b, uint64_t c) {
    const uint64_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// U[slot][b] += number of unsatisfied bonds (J S S' = -1) among the three
// forward bonds (+x, +y, +tau) of every site; each bond is counted once and
// E = -(3N - 2U) is the action of Eq. (Trotter-action).  A block covers one
// slot over kEnergyRun planes, four planes per block barrier; its planes
// stream through a ring of kEnergyBuf shared-memory planes filled by cp.async
// kEnergyAhead planes ahead, so every word is read from HBM once and the +x,
// +y and +tau neighbours come from shared memory.  A thread owns two adjacent
// site words of a row: six bond words per plane, 24 per step, summed per
// sample bit by a Harley-Seal carry-save tree whose ones, twos, fours,
// eights and sixteens are the low bit-planes of the thread's count (one
// ripple into the count of 32s per step); the warp then sums its counters
// with shuffles and one lane turns them into per-sample integers.
__global__ void __launch_bounds__(512, 2) k_energy(Group g) {
    extern __shared__ __align__(16) uint64_t eplanes[];  // [kEnergyBuf][L^2]
    __shared__ int cnt[64];
    const int s = blockIdx.x;
    const int L = g.L, L2 = L * L, Lt = g.Ltau;
    const int w = s / (g.R * g.K);
    const uint64_t *S = g.S + (size_t)s * g.N;
    for (int b = threadIdx.x; b < 64; b += blockDim.x) cnt[b] = 0;
    const int t0 = blockIdx.y * kEnergyRun, t1 = min(t0 + kEnergyRun, Lt);
    const int xy = 2 * (int)threadIdx.x;
    const bool own = xy < L2;  // sites xy and xy + 1 (L is even: one row)
    // plane q of the block (t0 <= q <= t1; q = Lt is plane 0) into ring slot q % kEnergyBuf
    auto issue = [&](int q) {
        if (own && q <= t1) {
            const int gq = q == Lt ? 0 : q;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(eplanes + (size_t)(q % kEnergyBuf) * L2 + xy);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(S + (size_t)gq * L2 + xy)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    uint64_t c[kEnergyPlanes];
#pragma unroll
    for (int p = 0; p < kEnergyPlanes; ++p) c[p] = 0;
    int xr = 0, yu = 0;
    uint64_t j0x = 0, j1x = 0, j0y = 0, j1y = 0;
    if (own) {
        const int y = xy / L, x = xy - y * L;  // x even, x + 1 < L
        xr = y * L + (x + 2 == L ? 0 : x + 2);  // right neighbour of site xy + 1
        yu = (y + 1 == L ? 0 : y + 1) * L + x;  // up neighbours: yu, yu + 1
        j0x = g.Jx[(size_t)w * L2 + xy];
        j1x = g.Jx[(size_t)w * L2 + xy + 1];
        j0y = g.Jy[(size_t)w * L2 + xy];
        j1y = g.Jy[(size_t)w * L2 + xy + 1];
    }
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;
#pragma unroll
    for (int d = 0; d <= kEnergyAhead; ++d) issue(t0 + d);
    // the six bond words of the thread's two sites on plane q (zero past t1)
    auto bonds = [&](int q, uint64_t (&x)[6]) {
        if (q >= t1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) x[k] = 0;
            return;
        }
        const uint64_t *P = eplanes + (size_t)(q % kEnergyBuf) * L2;
        const uint64_t *Pn = eplanes + (size_t)((q + 1) % kEnergyBuf) * L2;
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(P + xy);
        const ulonglong2 u = *reinterpret_cast<const ulonglong2 *>(P + yu);
        const ulonglong2 n = *reinterpret_cast<const ulonglong2 *>(Pn + xy);
        const uint64_t r1 = P[xr];
        const uint64_t ft = q + 1 == Lt ? apbc : 0ull;
        x[0] = v.x ^ v.y ^ j0x;
        x[1] = v.x ^ u.x ^ j0y;
        x[2] = v.x ^ n.x ^ ft;
        x[3] = v.y ^ r1 ^ j1x;
        x[4] = v.y ^ u.y ^ j1y;
        x[5] = v.y ^ n.y ^ ft;
    };
    uint64_t ones = 0, twos = 0, fours = 0, eights = 0, sixteens = 0;
    // 12 bond words into ones / twos / fours; the two carries of weight 8 out
    auto tree12 = [&](const uint64_t (&x)[6], const uint64_t (&y)[6], uint64_t &eA, uint64_t &eB) {
        uint64_t tA, tB, tC, tD, tE, tF, fA, fB, fC;
        csa(tA, ones, ones, x[0], x[1]);
        csa(tB, ones, ones, x[2], x[3]);
        csa(fA, twos, twos, tA, tB);
        csa(tC, ones, ones, x[4], x[5]);
        csa(tD, ones, ones, y[0], y[1]);
        csa(fB, twos, twos, tC, tD);
        csa(eA, fours, fours, fA, fB);
        csa(tE, ones, ones, y[2], y[3]);
        csa(tF, ones, ones, y[4], y[5]);
        csa(fC, twos, twos, tE, tF);
        eB = fours & fC;
        fours ^= fC;
    };
    for (int q = t0; q < t1; q += 4) {
        // planes q .. q + 4 have landed (q + 5 .. q + kEnergyAhead may be in flight)
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kEnergyAhead - 4) : "memory");
        __syncthreads();
        // the slots of planes q - 4 .. q - 1 are free for every thread: refill them
        issue(q + kEnergyAhead + 1);
        issue(q + kEnergyAhead + 2);
        issue(q + kEnergyAhead + 3);
        issue(q + kEnergyAhead + 4);
        if (own) {
            uint64_t x[6], y[6], eA1, eB1, eA2, eB2;
            bonds(q, x);
            bonds(q + 1, y);
            tree12(x, y, eA1, eB1);
            bonds(q + 2, x);
            bonds(q + 3, y);
            tree12(x, y, eA2, eB2);
            uint64_t s16a, s16b, c32;
            csa(s16a, eights, eights, eA1, eB1);
            csa(s16b, eights, eights, eA2, eB2);
            csa(c32, sixteens, sixteens, s16a, s16b);
            // count of 32s += c32 (a thread counts at most 6 x kEnergyRun < 2^10)
            uint64_t carry = c32;
#pragma unroll
            for (int p = 0; p < kEnergyThirtyTwos; ++p) {
                const uint64_t t = c[p] & carry;
                c[p] ^= carry;
                carry = t;
            }
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    // the thread's count: ones .. sixteens, then the 32s
#pragma unroll
    for (int p = kEnergyPlanes - 1; p >= 5; --p) c[p] = c[p - 5];
    c[0] = ones;
    c[1] = twos;
    c[2] = fours;
    c[3] = eights;
    c[4] = sixteens;
    // warp sum of the bitsliced counters (at most 32 * 6 * kEnergyRun < 2^15)
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t other[kEnergyPlanes];
#pragma unroll
        for (int p = 0; p < kEnergyPlanes; ++p) other[p] = __shfl_down_sync(0xffffffffu, c[p], o);
        vadd_counter(c, other);
    }
    // lane l turns sample bits l and l + 32 of lane 0's counter into integers
    {
        const int lane = threadIdx.x & 31;
        int v0 = 0, v1 = 0;
#pragma unroll
        for (int p = 0; p < kEnergyPlanes; ++p) {
            const uint64_t cp = __shfl_sync(0xffffffffu, c[p], 0);
            v0 |= (int)((cp >> lane) & 1ull) << p;
            v1 |= (int)((cp >> (lane + 32)) & 1ull) << p;
        }
        if (v0) atomicAdd(&cnt[lane], v0);
        if (v1) atomicAdd(&cnt[lane + 32], v1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 64; b += blockDim.x)
        if (cnt[b]) atomicAdd(&g.U[(size_t)s * 64 + b], cnt[b]);
}

cudaError_t launch_energy(const Group &g, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g.U, 0, sizeof(int32_t) * (size_t)g.nslots * 64, st);
    if (e != cudaSuccess) return e;
    // one thread per two site words; a ring of kEnergyBuf planes in shared memory
    const int L2 = g.L * g.L;
    const int threads = (L2 / 2 + 31) / 32 * 32;
    const size_t sm = (size_t)kEnergyBuf * L2 * sizeof(uint64_t);
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(k_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(g.nslots, (g.Ltau + kEnergyRun - 1) / kEnergyRun);
    count_launches(1);
    k_energy<<<grid, threads, sm, st>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Parallel tempering.  One block per (word-group w, replica r), one thread per
// sample bit.  Pairs (k_i, k_i+1) are tried in increasing i with the actions
// left by earlier swaps of the same step.  A swap of sample b exchanges the
// configurations held at ladder positions i and i+1; here it is recorded as
// bit b of a per-pair mask and applied to the spin words by k_pt_apply.
// ---------------------------------------------------------------------------
constexpr int kMaxK = 128;

__global__ void __launch_bounds__(64) k_pt_decide(Group g, uint32_t m, uint32_t k0, uint32_t k1) {
    const int wr = blockIdx.x, b = threadIdx.x;
    const int w = wr / g.R;
    const int K = g.K;
    const long long three_n = 3LL * g.N;
    long long E[kMaxK];
    for (int j = 0; j < K; ++j) E[j] = 2LL * g.U[((size_t)wr * K + j) * 64 + b] - three_n;
    const uint32_t tag = (STREAM_PT << 24) | ((uint32_t)g.gid << 8);
    for (int i = 0; i + 1 < K; ++i) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(i * 16 + b / 4), m, (uint32_t)wr, tag), k0, k1);
        const uint32_t u = pick(r, b & 3);
        bool accept;
        if (E[i + 1] >= E[i]) {
            accept = true;
        } else {
            const long long n = E[i] - E[i + 1];
            if ((n >> 6) >= g.ptA_len[i]) {
                accept = false;
            } else {
                const unsigned long long thr =
                    (g.ptA[g.ptA_off[i] + (n >> 6)] * g.ptB[i * 64 + (n & 63)]) >> 32;
                accept = (unsigned long long)u < thr;
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, accept);
        if ((b & 31) == 0) g.swapmask[((size_t)wr * (K - 1) + i) * 2 + (b >> 5)] = ball;
        if (accept) {
            const long long tmp = E[i];
            E[i] = E[i + 1];
            E[i + 1] = tmp;
            atomicAdd(&g.acc[((size_t)w * 64 + b) * (K - 1) + i], 1ull);
        }
    }
    for (int j = 0; j < K; ++j) g.U[((size_t)wr * K + j) * 64 + b] = (int32_t)((E[j] + three_n) / 2);
}

// Apply the swaps of one tempering step to the spin words: for every site of
// every (w, r), walk the ladder and exchange the masked bits of positions i
// and i+1 in the same order as the decisions.
__global__ void k_pt_apply(Group g) {
    constexpr int B = 8;  // slots loaded together (independent loads in flight)
    const int K = g.K;
    const size_t total = (size_t)g.W * g.R * g.N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t wr = idx / g.N, n = idx % g.N;
        const uint32_t *M = g.swapmask + wr * (K - 1) * 2;
        uint64_t *base = g.S + wr * K * (size_t)g.N + n;
        // cur: slot i0 after the swaps of pairs < i0 (cur0: as loaded)
        uint64_t cur = base[0], cur0 = cur;
        for (int i0 = 0; i0 + 1 < K; i0 += B) {
            const int nb = min(B, K - 1 - i0);  // pairs i0 .. i0 + nb - 1, slots i0 + 1 .. i0 + nb
            uint64_t msk[B];
            uint64_t any = 0;
#pragma unroll
            for (int k = 0; k < B; ++k) {
                msk[k] = k < nb ? ((uint64_t)__ldg(&M[2 * (i0 + k)]) | ((uint64_t)__ldg(&M[2 * (i0 + k) + 1]) << 32)) : 0ull;
                any |= msk[k];
            }
            if (!any) {
                // no swap among these pairs: slots i0 + 1 .. i0 + nb keep their bits
                if (cur != cur0) base[(size_t)i0 * g.N] = cur;
                cur = cur0 = base[(size_t)(i0 + nb) * g.N];
                continue;
            }
            uint64_t v[B];
#pragma unroll
            for (int k = 0; k < B; ++k)
                if (k < nb) v[k] = base[(size_t)(i0 + 1 + k) * g.N];
#pragma unroll
            for (int k = 0; k < B; ++k) {
                if (k < nb) {
                    uint64_t nxt = v[k];
                    const uint64_t nxt0 = nxt;
                    const uint64_t d = (cur ^ nxt) & msk[k];
                    cur ^= d;
                    nxt ^= d;
                    if (cur != cur0) base[(size_t)(i0 + k) * g.N] = cur;
                    cur = nxt;
                    cur0 = nxt0;
                }
            }
        }
        if (cur != cur0) base[(size_t)(K - 1) * g.N] = cur;
    }
}

cudaError_t launch_tempering(const Group &g, uint32_t m, uint64_t seed, cudaStream_t st) {
    if (g.K < 2) return cudaSuccess;
    count_launches(1);
    k_pt_decide<<<g.W * g.R, 64, 0, st>>>(g, m, (uint32_t)seed, (uint32_t)(seed >> 32));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t total = (size_t)g.W * g.R * g.N;
    long long blocks = (long long)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    count_launches(1);
    k_pt_apply<<<(int)blocks, 256, 0, st>>>(g);
    return cudaGetLastError();
}

}  // namespace qsg
