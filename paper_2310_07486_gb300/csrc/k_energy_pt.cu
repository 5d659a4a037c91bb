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

// k_energy with L compiled in (the lattice sizes of the sweep's fixed-L
// kernels and the smaller even sizes of the ragged workloads).  The same
// count, in a leaner loop: each step's four planes come in one cp.async group
// and the four refill copies use constant offsets; a thread keeps its own two
// words of the next plane (they are the +tau neighbours of this one) in
// registers, so a plane costs three shared-memory loads; only a step that
// runs past the block's last plane takes the per-plane checks; every plane
// index of the ring is fixed by the step's first plane.
template <int L>
__host__ __device__ constexpr int energy_threads() {
    return (L * L / 2 + 31) / 32 * 32;
}

template <int L, int RUN>
__global__ void __launch_bounds__(energy_threads<L>(), 3) k_energy_l(Group g) {
    constexpr int L2 = L * L;
    constexpr int kT = energy_threads<L>();
    constexpr int kThirty = RUN <= 128 ? 5 : 6;            // planes of the count of 32s (6 RUN / 32 < 2^kThirty)
    constexpr int kPlanes = RUN <= 128 ? 15 : 16;          // bits of a warp's count (32 x 6 x RUN < 2^kPlanes)
    static_assert(RUN % 4 == 0 && RUN <= 256, "run of planes");
    extern __shared__ __align__(16) uint64_t ring[];       // [kEnergyBuf][L2]
    __shared__ int cnt[64];
    const int s = blockIdx.x;
    const int Lt = g.Ltau;
    const int t0 = blockIdx.y * RUN, t1 = min(t0 + RUN, Lt);
    const int tid = threadIdx.x;
    for (int b = tid; b < 64; b += kT) cnt[b] = 0;
    const int xy = 2 * tid;
    const bool own = xy < L2;  // sites xy and xy + 1 (L is even: one row)
    const int y = xy / L, x = xy - (xy / L) * L;
    const int xr = y * L + (x + 2 == L ? 0 : x + 2);      // right neighbour of site xy + 1
    const int yu = (y + 1 == L ? 0 : y + 1) * L + x;       // up neighbours: yu, yu + 1
    const int w = s / (g.R * g.K);
    const uint64_t *Sx = g.S + (size_t)s * g.N + xy;       // the thread's column of words
    const unsigned ring0 = (unsigned)__cvta_generic_to_shared(ring) + 8u * (unsigned)xy;
    uint64_t j0x = 0, j1x = 0, j0y = 0, j1y = 0;
    if (own) {
        j0x = g.Jx[(size_t)w * L2 + xy];
        j1x = g.Jx[(size_t)w * L2 + xy + 1];
        j0y = g.Jy[(size_t)w * L2 + xy];
        j1y = g.Jy[(size_t)w * L2 + xy + 1];
    }
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;
    auto copy = [&](int q, int gq) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(ring0 + 8u * (unsigned)((q % kEnergyBuf) * L2)),
                     "l"(Sx + (size_t)gq * L2)
                     : "memory");
    };
    // planes q .. q + 3 (those up to t1; plane Lt is plane 0) as one group
    auto issue4 = [&](int q) {
        if (own) {
            if (q + 3 <= t1 && q + 3 < Lt) {
                const unsigned d = ring0 + 8u * (unsigned)((q % kEnergyBuf) * L2);
                const uint64_t *src = Sx + (size_t)q * L2;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 8u * i * L2), "l"(src + i * L2)
                                 : "memory");
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (q + i <= t1) copy(q + i, q + i == Lt ? 0 : q + i);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    issue4(t0);
    issue4(t0 + 4);
    issue4(t0 + 8);
    uint64_t ones = 0, twos = 0, fours = 0, eights = 0, sixteens = 0;
    uint64_t c32[kThirty];
#pragma unroll
    for (int p = 0; p < kThirty; ++p) c32[p] = 0;
    ulonglong2 v = make_ulonglong2(0ull, 0ull);  // the thread's words of the current plane
    // the six bond words of plane P (next plane Pn); v moves on to the next plane
    auto bonds = [&](const uint64_t *P, const uint64_t *Pn, uint64_t ft, uint64_t (&b)[6]) {
        const ulonglong2 u = *reinterpret_cast<const ulonglong2 *>(P + yu);
        const uint64_t r1 = P[xr];
        const ulonglong2 n = *reinterpret_cast<const ulonglong2 *>(Pn + xy);
        b[0] = v.x ^ v.y ^ j0x;
        b[1] = v.x ^ u.x ^ j0y;
        b[2] = v.x ^ n.x ^ ft;
        b[3] = v.y ^ r1 ^ j1x;
        b[4] = v.y ^ u.y ^ j1y;
        b[5] = v.y ^ n.y ^ ft;
        v = n;
    };
    auto tree12 = [&](const uint64_t (&a)[6], const uint64_t (&b)[6], uint64_t &eA, uint64_t &eB) {
        uint64_t tA, tB, tC, tD, tE, tF, fA, fB, fC;
        csa(tA, ones, ones, a[0], a[1]);
        csa(tB, ones, ones, a[2], a[3]);
        csa(fA, twos, twos, tA, tB);
        csa(tC, ones, ones, a[4], a[5]);
        csa(tD, ones, ones, b[0], b[1]);
        csa(fB, twos, twos, tC, tD);
        csa(eA, fours, fours, fA, fB);
        csa(tE, ones, ones, b[2], b[3]);
        csa(tF, ones, ones, b[4], b[5]);
        csa(fC, twos, twos, tE, tF);
        eB = fours & fC;
        fours ^= fC;
    };
    auto ripple = [&](uint64_t carry) {  // count of 32s += carry
#pragma unroll
        for (int p = 0; p < kThirty; ++p) {
            const uint64_t t = c32[p] & carry;
            c32[p] ^= carry;
            carry = t;
        }
    };
    int q = t0;
    for (; q + 4 <= t1; q += 4) {
        // planes q .. q + 4 have landed (the group of q + 8 .. q + 11 may be in flight)
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        // the slots of planes q - 4 .. q - 1 are free for every thread: refill them
        issue4(q + 12);
        if (own) {
            const uint64_t *P = ring + (q % kEnergyBuf) * L2;
            if (q == t0) v = *reinterpret_cast<const ulonglong2 *>(P + xy);
            // only the last of the four planes can close the tau ring
            const uint64_t ft3 = q + 4 == Lt ? apbc : 0ull;
            uint64_t a[6], b[6], eA1, eB1, eA2, eB2;
            bonds(P, P + L2, 0ull, a);
            bonds(P + L2, P + 2 * L2, 0ull, b);
            tree12(a, b, eA1, eB1);
            bonds(P + 2 * L2, P + 3 * L2, 0ull, a);
            bonds(P + 3 * L2, ring + ((q + 4) % kEnergyBuf) * L2, ft3, b);
            tree12(a, b, eA2, eB2);
            uint64_t s16a, s16b, carry;
            csa(s16a, eights, eights, eA1, eB1);
            csa(s16b, eights, eights, eA2, eB2);
            csa(carry, sixteens, sixteens, s16a, s16b);
            ripple(carry);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (q < t1) {
        // two planes left (runs and L_tau are even)
        __syncthreads();
        if (own) {
            const uint64_t *P = ring + (q % kEnergyBuf) * L2;
            if (q == t0) v = *reinterpret_cast<const ulonglong2 *>(P + xy);
            uint64_t a[6], b[6], eA1, eB1;
            bonds(P, ring + ((q + 1) % kEnergyBuf) * L2, 0ull, a);
            bonds(ring + ((q + 1) % kEnergyBuf) * L2, ring + ((q + 2) % kEnergyBuf) * L2, q + 2 == Lt ? apbc : 0ull, b);
            tree12(a, b, eA1, eB1);
            uint64_t s16a;
            csa(s16a, eights, eights, eA1, eB1);
            const uint64_t carry = sixteens & s16a;
            sixteens ^= s16a;
            ripple(carry);
        }
    }
    // the thread's count: ones .. sixteens, then the 32s
    uint64_t c[kPlanes];
    c[0] = ones;
    c[1] = twos;
    c[2] = fours;
    c[3] = eights;
    c[4] = sixteens;
#pragma unroll
    for (int p = 5; p < kPlanes; ++p) c[p] = p - 5 < kThirty ? c32[p - 5 < kThirty ? p - 5 : 0] : 0ull;
    // warp sum of the bitsliced counters; after the round with offset o a
    // lane's count is below 6 RUN (32 / o), so fewer planes need adding
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int o = 16 >> r;
        constexpr int base = 5 + kThirty;  // planes of one thread's count
        uint64_t carry = 0;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            if (p < base + r + 1) {
                const uint64_t other = __shfl_down_sync(0xffffffffu, c[p], o);
                const uint64_t sum = c[p] ^ other ^ carry;
                carry = (c[p] & other) | (carry & (c[p] ^ other));
                c[p] = sum;
            }
        }
    }
    {
        const int lane = tid & 31;
        int v0 = 0, v1 = 0;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const uint64_t cp = __shfl_sync(0xffffffffu, c[p], 0);
            v0 |= (int)((cp >> lane) & 1ull) << p;
            v1 |= (int)((cp >> (lane + 32)) & 1ull) << p;
        }
        if (v0) atomicAdd(&cnt[lane], v0);
        if (v1) atomicAdd(&cnt[lane + 32], v1);
    }
    __syncthreads();
    for (int b = tid; b < 64; b += kT)
        if (cnt[b]) atomicAdd(&g.U[(size_t)s * 64 + b], cnt[b]);
}

template <int L, int RUN>
static cudaError_t launch_energy_l(const Group &g, cudaStream_t st) {
    constexpr size_t sm = (size_t)kEnergyBuf * L * L * sizeof(uint64_t);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_energy_l<L, RUN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(g.nslots, (g.Ltau + RUN - 1) / RUN);
    count_launches(1);
    k_energy_l<L, RUN><<<grid, energy_threads<L>(), sm, st>>>(g);
    return cudaGetLastError();
}

static cudaError_t launch_energy_generic(const Group &g, cudaStream_t st) {
    // one thread per two site words; a ring of kEnergyBuf planes in shared memory
    const int L2 = g.L * g.L;
    const int threads = (L2 / 2 + 31) / 32 * 32;
    const size_t sm = (size_t)kEnergyBuf * L2 * sizeof(uint64_t);
    if (sm > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(g.nslots, (g.Ltau + kEnergyRun - 1) / kEnergyRun);
    count_launches(1);
    k_energy<<<grid, threads, sm, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_energy(const Group &g, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g.U, 0, sizeof(int32_t) * (size_t)g.nslots * 64, st);
    if (e != cudaSuccess) return e;
    // runs of 256 planes halve the final warp sums per word where L_tau
    // leaves enough blocks (4.5 waves of 456 resident blocks at the 256-slot
    // L = 24, L_tau = 2048 state: 0.55 -> 0.52 ms)
    const bool long_runs = g.Ltau >= 1024;
    switch (g.L) {
        case 8: return long_runs ? launch_energy_l<8, 256>(g, st) : launch_energy_l<8, 128>(g, st);
        case 12: return long_runs ? launch_energy_l<12, 256>(g, st) : launch_energy_l<12, 128>(g, st);
        case 16: return long_runs ? launch_energy_l<16, 256>(g, st) : launch_energy_l<16, 128>(g, st);
        case 20: return long_runs ? launch_energy_l<20, 256>(g, st) : launch_energy_l<20, 128>(g, st);
        case 24: return long_runs ? launch_energy_l<24, 256>(g, st) : launch_energy_l<24, 128>(g, st);
        default: return launch_energy_generic(g, st);
    }
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

// Apply the swaps of one tempering step to the spin words.  A block serves
// one (w, r) and a range of sites; it first lists the ladder pairs whose swap
// mask is not zero (the same for all its sites), and every thread then walks
// only those pairs in increasing order, exchanging the masked bits of
// positions i and i + 1 as the decisions did.  Consecutive listed pairs form
// a chain (a configuration can move several positions in one step); a slot is
// read only when a listed pair touches it and written only when its bits
// changed.  Slots are loaded for eight listed pairs at a time (independent
// loads in flight).
constexpr int kApplyThreads = 256;

__global__ void __launch_bounds__(kApplyThreads) k_pt_apply(Group g) {
    constexpr int B = 8;
    __shared__ uint64_t msk[kMaxK];
    __shared__ int act[kMaxK];
    __shared__ int nact;
    const int K = g.K, N = g.N;
    for (int wr = blockIdx.y; wr < g.W * g.R; wr += gridDim.y) {
        const uint32_t *M = g.swapmask + (size_t)wr * (K - 1) * 2;
        if (threadIdx.x < 32) {
            // warp 0 lists the pairs with a swap, in increasing order
            int n0 = 0;
            for (int i0 = 0; i0 + 1 < K; i0 += 32) {
                const int i = i0 + (int)threadIdx.x;
                uint64_t m = 0;
                if (i + 1 < K) m = (uint64_t)M[2 * i] | ((uint64_t)M[2 * i + 1] << 32);
                const unsigned ball = __ballot_sync(0xffffffffu, m != 0);
                if (m) {
                    const int at = n0 + __popc(ball & ((1u << threadIdx.x) - 1u));
                    act[at] = i;
                    msk[at] = m;
                }
                n0 += __popc(ball);
            }
            if (threadIdx.x == 0) nact = n0;
        }
        __syncthreads();
        const int na = nact;
        uint64_t *const slot0 = g.S + (size_t)wr * K * N;
        for (int n = blockIdx.x * kApplyThreads + threadIdx.x; na > 0 && n < N; n += gridDim.x * kApplyThreads) {
            uint64_t *base = slot0 + n;
            uint64_t cur = 0, cur0 = 0;  // slot prev + 1 after the swaps so far, and as loaded
            int prev = -2;               // the last pair walked
            for (int a0 = 0; a0 < na; a0 += B) {
                const int nb = min(B, na - a0);
                uint64_t vn[B], vs[B];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    if (k < nb) {
                        const int p = act[a0 + k], pp = k == 0 ? prev : act[a0 + k - 1];
                        vn[k] = base[(size_t)(p + 1) * N];
                        vs[k] = p != pp + 1 ? base[(size_t)p * N] : 0ull;  // a chain starts at p
                    }
                }
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    if (k < nb) {
                        const int p = act[a0 + k], pp = k == 0 ? prev : act[a0 + k - 1];
                        if (p != pp + 1) {
                            if (pp >= 0 && cur != cur0) base[(size_t)(pp + 1) * N] = cur;
                            cur = cur0 = vs[k];
                        }
                        uint64_t nxt = vn[k];
                        const uint64_t nxt0 = nxt;
                        const uint64_t d = (cur ^ nxt) & msk[a0 + k];
                        cur ^= d;
                        nxt ^= d;
                        if (cur != cur0) base[(size_t)p * N] = cur;
                        cur = nxt;
                        cur0 = nxt0;
                    }
                }
                prev = act[a0 + nb - 1];
            }
            if (na > 0 && cur != cur0) base[(size_t)(prev + 1) * N] = cur;
        }
        __syncthreads();  // the list is rebuilt for the next (w, r)
    }
}

static cudaError_t launch_apply(const Group &g, cudaStream_t st);

cudaError_t launch_tempering(const Group &g, uint32_t m, uint64_t seed, cudaStream_t st) {
    if (g.K < 2) return cudaSuccess;
    count_launches(1);
    k_pt_decide<<<g.W * g.R, 64, 0, st>>>(g, m, (uint32_t)seed, (uint32_t)(seed >> 32));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_apply(g, st);
}

static cudaError_t launch_apply(const Group &g, cudaStream_t st) {
    // one resident wave of blocks (2048 threads per SM) shared out over the
    // (w, r) rows; a block strides over its row's sites
    const int wr = g.W * g.R;
    long long bx = (152LL * 2048 / kApplyThreads + wr - 1) / wr;
    const long long need = (g.N + kApplyThreads - 1) / kApplyThreads;
    if (bx > need) bx = need;
    if (bx < 1) bx = 1;
    count_launches(1);
    k_pt_apply<<<dim3((unsigned)bx, (unsigned)(wr < 65535 ? wr : 65535)), kApplyThreads, 0, st>>>(g);
    return cudaGetLastError();
}

}  // namespace qsg
