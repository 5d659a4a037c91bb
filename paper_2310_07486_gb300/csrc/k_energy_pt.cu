// k_energy_pt.cu -- integer action of every configuration and the
// parallel-tempering step over the k ladder (Methods, "Simulation details").
#include "qsg_launch.h"

namespace qsg {

// Add one word to a bitsliced vertical counter (plane p holds bit p of the
// per-position counts); the carry chain stops as soon as no position carries.
template <int P>
__device__ __forceinline__ void vadd(uint64_t (&c)[P], uint64_t x) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const uint64_t t = c[p] & x;
        c[p] ^= x;
        x = t;
        if (!x) break;
    }
}

constexpr int kEnergyPlanes = 16;
constexpr int kEnergyThreads = 256;

// U[slot][b] += number of unsatisfied bonds (J S S' = -1) among the three
// forward bonds (+x, +y, +tau) of every site in this block's chunk.  Each bond
// is counted once; E = -(3N - 2U) is the action of Eq. (Trotter-action).
__global__ void __launch_bounds__(kEnergyThreads) k_energy(Group g, int sites_per_block) {
    __shared__ int cnt[64];
    const int s = blockIdx.y;
    const int L = g.L, L2 = L * L, Lt = g.Ltau;
    const int w = s / (g.R * g.K);
    const uint64_t *S = g.S + (size_t)s * g.N;
    const uint64_t *Jx = g.Jx + (size_t)w * L2, *Jy = g.Jy + (size_t)w * L2;
    if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
    __syncthreads();
    uint64_t c[kEnergyPlanes];
#pragma unroll
    for (int p = 0; p < kEnergyPlanes; ++p) c[p] = 0;
    const int n0 = blockIdx.x * sites_per_block;
    const int n1 = min(n0 + sites_per_block, g.N);
    for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        const int t = n / L2, xy = n % L2, y = xy / L, x = xy % L;
        const uint64_t v = S[n];
        const uint64_t vx = S[t * L2 + y * L + (x + 1 == L ? 0 : x + 1)];
        const uint64_t vy = S[t * L2 + (y + 1 == L ? 0 : y + 1) * L + x];
        const uint64_t vt = S[(t + 1 == Lt ? 0 : t + 1) * L2 + xy];
        const uint64_t ft = (g.boundary == 1 && t == Lt - 1) ? ~0ull : 0ull;
        vadd(c, v ^ vx ^ Jx[xy]);
        vadd(c, v ^ vy ^ Jy[xy]);
        vadd(c, v ^ vt ^ ft);
    }
    for (int b = 0; b < 64; ++b) {
        int v = 0;
#pragma unroll
        for (int p = 0; p < kEnergyPlanes; ++p) v |= (int)((c[p] >> b) & 1ull) << p;
        if (v) atomicAdd(&cnt[b], v);
    }
    __syncthreads();
    if (threadIdx.x < 64) atomicAdd(&g.U[(size_t)s * 64 + threadIdx.x], cnt[threadIdx.x]);
}

cudaError_t launch_energy(const Group &g, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g.U, 0, sizeof(int32_t) * (size_t)g.nslots * 64, st);
    if (e != cudaSuccess) return e;
    // <= 3 * 64 * 256 bonds per thread keeps every count below 2^16
    const int spb = kEnergyThreads * 64;
    dim3 grid((g.N + spb - 1) / spb, g.nslots);
    count_launches(1);
    k_energy<<<grid, kEnergyThreads, 0, st>>>(g, spb);
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
    const int K = g.K;
    const size_t total = (size_t)g.W * g.R * g.N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t wr = idx / g.N, n = idx % g.N;
        const uint32_t *M = g.swapmask + wr * (K - 1) * 2;
        uint64_t *base = g.S + wr * K * (size_t)g.N + n;
        uint64_t cur = base[0], cur0 = cur;
        for (int i = 0; i + 1 < K; ++i) {
            const uint64_t msk = (uint64_t)M[2 * i] | ((uint64_t)M[2 * i + 1] << 32);
            uint64_t nxt = base[(size_t)(i + 1) * g.N];
            const uint64_t nxt0 = nxt;
            const uint64_t d = (cur ^ nxt) & msk;
            cur ^= d;
            nxt ^= d;
            if (cur != cur0) base[(size_t)i * g.N] = cur;
            cur = nxt;
            cur0 = nxt0;
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
