// qsg_sweep.cuh -- device pieces shared by the sweep kernels (k_wavefront.cu,
// k_sweep_unit.cu): the shared-memory plane ring, the threshold search and the
// bitsliced site update on multispin words.
#pragma once
#include "qsg_device.cuh"

namespace qsg {
namespace sweep {

constexpr int kRing = 16;  // planes held in shared memory (a power of two)

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

struct Thresh {
    uint32_t t[7];  // Metropolis: t[0..2]; heat bath: t[0..6]; non-increasing
};

// Bits of the scalar threshold m that the bitsliced count is compared with,
// as all-ones / all-zero masks, found by a binary search over the monotone
// table.  Heat bath: m = #{n : u < T[n]} (S = -1 iff n_neg >= m).
// Metropolis: m = 3 - #{c : u < T[c]} (flip iff n_unsat >= m).
template <int ALGO>
__device__ __forceinline__ void threshold_masks(uint32_t u, const Thresh &T, uint32_t &m0, uint32_t &m1,
                                                uint32_t &m2) {
    if (ALGO == 0) {
        const bool a1 = u < T.t[1];
        const bool a0 = u < (a1 ? T.t[2] : T.t[0]);
        m2 = 0u;
        m1 = a1 ? 0u : ~0u;
        m0 = a0 ? 0u : ~0u;
    } else {
        const bool c2 = u < T.t[3];
        const bool c1 = u < (c2 ? T.t[5] : T.t[1]);
        const uint32_t t0 = c1 ? (c2 ? T.t[6] : T.t[2]) : (c2 ? T.t[4] : T.t[0]);
        const bool c0 = u < t0;
        m2 = c2 ? ~0u : 0u;
        m1 = c1 ? ~0u : 0u;
        m0 = c0 ? ~0u : 0u;
    }
}

__device__ __forceinline__ uint64_t widen(uint32_t m) { return ((uint64_t)m << 32) | m; }

// One site update on multispin words.  Terms: nr/nl/nu/nd spatial neighbours
// with couplings jr/jl/ju/jd, ntp/ntm time neighbours (APBC sign folded in).
// b = the number of the six terms a_i (neighbour XOR coupling) that are 1.
// Heat bath: the new spin is [b >= m].  Metropolis: with c the old spin the
// unsatisfied bonds number b (c = 0) or 6 - b (c = 1), and the spin flips iff
// that count is >= m; so the new spin is [b >= m] for c = 0 and
// [6 - b < m] = [b >= 7 - m] for c = 1, and 7 - m = m XOR 7 for m <= 7: one
// comparison [b >= m XOR 7c] with a threshold that differs per sample bit.
template <int ALGO>
__device__ __forceinline__ uint64_t update_site(uint64_t c, uint64_t nr, uint64_t nl, uint64_t nu, uint64_t nd,
                                                uint64_t ntp, uint64_t ntm, uint64_t jr, uint64_t jl, uint64_t ju,
                                                uint64_t jd, uint32_t u, const Thresh &T) {
    uint64_t b0, b1, b2;
    uint32_t m0, m1, m2;
    threshold_masks<ALGO>(u, T, m0, m1, m2);
    count6(nr ^ jr, nl ^ jl, nu ^ ju, nd ^ jd, ntp, ntm, b0, b1, b2);
    if (ALGO == 0) {  // m <= 3: bit 2 of the threshold is c itself
        const uint64_t t1 = widen(m1) ^ c;
        const uint64_t e0 = b0 | ~(widen(m0) ^ c);
        const uint64_t e1 = (b1 & ~t1) | (~(b1 ^ t1) & e0);
        return (b2 & ~c) | (~(b2 ^ c) & e1);
    }
    const uint64_t M0 = widen(m0), M1 = widen(m1), M2 = widen(m2);
    const uint64_t e0 = b0 | ~M0;
    const uint64_t e1 = (b1 & ~M1) | (~(b1 ^ M1) & e0);
    return (b2 & ~M2) | (~(b2 ^ M2) & e1);
}

}  // namespace sweep
}  // namespace qsg
