// k_init_sweep.cu -- instance generation, hot start and the one-thread-per-site
// checkerboard sweep (the plain reference form of the update; the fused
// wavefront kernel lives in k_wavefront.cu and produces the same bits).
#include "qsg_launch.h"

namespace qsg {

// Couplings J = +-1 with probability 1/2 for every sample and bond (Methods,
// "Model and simulations"): one Philox call per (word-group, direction, site).
__global__ void k_init_couplings(Group g, uint32_t k0, uint32_t k1) {
    const int L2 = g.L * g.L;
    const int total = g.W * 2 * L2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int n = i % L2, d = (i / L2) & 1, w = i / (2 * L2);
        const uint4 r = philox4x32_10(make_uint4((uint32_t)n, (uint32_t)d, (uint32_t)w,
                                                 (STREAM_J << 24) | ((uint32_t)g.gid << 8)), k0, k1);
        const uint64_t bits = (uint64_t)r.x | ((uint64_t)r.y << 32);
        (d == 0 ? g.Jx : g.Jy)[(size_t)w * L2 + n] = bits;
    }
}

// Hot start: every spin of every slot drawn from Philox stream INIT.
__global__ void k_init_spins(Group g, uint32_t k0, uint32_t k1) {
    const size_t total = (size_t)g.nslots * g.N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)(i % g.N), s = (uint32_t)(i / g.N);
        const uint4 r = philox4x32_10(make_uint4(n, 0u, s, (STREAM_INIT << 24) | ((uint32_t)g.gid << 8)), k0, k1);
        g.S[i] = (uint64_t)r.x | ((uint64_t)r.y << 32);
    }
}

// One colour of a checkerboard sweep, one thread per site word.  Sites of
// one colour never neighbour each other (L, L_tau even), so all of them update
// from the same state.
__global__ void k_half_sweep_ref(Group g, int colour, uint32_t sweep, uint32_t k0, uint32_t k1) {
    const int L = g.L, half = L / 2, Lt = g.Ltau;
    const long long per_slot = (long long)g.N / 2;
    const long long total = per_slot * g.nslots;
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / per_slot);
        const int m = (int)(i % per_slot);
        const int t = m / (L * half);
        const int rem = m % (L * half);
        const int y = rem / half, xh = rem % half;
        const int x = 2 * xh + ((y + t + colour) & 1);
        const int w = s / (g.R * g.K), j = s % g.K;
        uint64_t *S = g.S + (size_t)s * g.N;
        const int xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
        const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
        const int tp = t + 1 == Lt ? 0 : t + 1, tm = t == 0 ? Lt - 1 : t - 1;
        const size_t n = ((size_t)t * L + y) * L + x;
        uint64_t c = S[n];
        const uint64_t nxp = S[((size_t)t * L + y) * L + xp], nxm = S[((size_t)t * L + y) * L + xm];
        const uint64_t nyp = S[((size_t)t * L + yp) * L + x], nym = S[((size_t)t * L + ym) * L + x];
        const uint64_t ntp = S[((size_t)tp * L + y) * L + x], ntm = S[((size_t)tm * L + y) * L + x];
        const uint64_t *Jx = g.Jx + (size_t)w * L * L, *Jy = g.Jy + (size_t)w * L * L;
        const uint64_t jxp = Jx[y * L + x], jxm = Jx[y * L + xm], jyp = Jy[y * L + x], jym = Jy[ym * L + x];
        const uint64_t fp = (g.boundary == 1 && t == Lt - 1) ? ~0ull : 0ull;  // APBC wrap bond
        const uint64_t fm = (g.boundary == 1 && t == 0) ? ~0ull : 0ull;
        // column pairs start at x = y & 1 (so odd rows pair (1,2), ..., (L-1,0))
        const int xs = x - (y & 1) < 0 ? L - 1 : x - (y & 1);
        const uint32_t block = (uint32_t)(((t >> 1) * L + y) * half + (xs >> 1));
        const uint4 r = philox4x32_10(make_uint4(block, sweep, (uint32_t)s, tag), k0, k1);
        const uint32_t u = pick(r, (t & 1) * 2 + (xs & 1));
        const uint32_t *T = g.thr + j * 16;
        uint64_t b0, b1, b2;
        if (g.algo == 0) {
            // unsatisfied bonds: S J S_nb = -1  <=>  bit(S) ^ bit(J) ^ bit(S_nb) = 1
            count6(c ^ nxp ^ jxp, c ^ nxm ^ jxm, c ^ nyp ^ jyp, c ^ nym ^ jym, c ^ ntp ^ fp, c ^ ntm ^ fm, b0, b1, b2);
            // S h = 6 - 2 n_unsat; flip iff n_unsat >= 3 - #{c : u < T[c]}
            c ^= ge_scalar(b0, b1, b2, 3u - count_above3(u, T));
        } else {
            // negative terms of h: J S_nb = -1  <=>  bit(J) ^ bit(S_nb) = 1
            count6(nxp ^ jxp, nxm ^ jxm, nyp ^ jyp, nym ^ jym, ntp ^ fp, ntm ^ fm, b0, b1, b2);
            // S = +1 iff u < T[n_neg]  <=>  n_neg < #{n : u < T[n]}
            c = ge_scalar(b0, b1, b2, count_above7(u, T + 8));
        }
        S[n] = c;
    }
}

// Device-to-device copy of spin state in 16-byte words (the copy engines move
// device memory at a fraction of what the SMs' loads and stores reach).
__global__ void k_copy16(uint4 *__restrict__ dst, const uint4 *__restrict__ src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __ldcs(src + i);
}

cudaError_t launch_copy_words(uint64_t *dst, const uint64_t *src, size_t words, cudaStream_t st) {
    if (words == 0) return cudaSuccess;
    if ((((uintptr_t)dst | (uintptr_t)src) & 15u) != 0 || (words & 1u) != 0)
        return cudaMemcpyAsync(dst, src, words * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    count_launches(1);
    k_copy16<<<152 * 8, 512, 0, st>>>(reinterpret_cast<uint4 *>(dst), reinterpret_cast<const uint4 *>(src), words / 2);
    return cudaGetLastError();
}

// Device copy of the sweep counter used by replayed graphs: set from the host
// value before the first replay, advanced by the last node of each replay.
__global__ void k_set_word(uint32_t *p, uint32_t v, int add) { *p = add ? *p + v : v; }

cudaError_t launch_set_word(uint32_t *p, uint32_t value, cudaStream_t st) {
    count_launches(1);
    k_set_word<<<1, 1, 0, st>>>(p, value, 0);
    return cudaGetLastError();
}

cudaError_t launch_add_word(uint32_t *p, uint32_t value, cudaStream_t st) {
    count_launches(1);
    k_set_word<<<1, 1, 0, st>>>(p, value, 1);
    return cudaGetLastError();
}

static int grid_for(long long work, int block) {
    long long g = (work + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_init_couplings(const Group &g, uint64_t seed, cudaStream_t st) {
    const int total = g.W * 2 * g.L * g.L;
    count_launches(1);
    k_init_couplings<<<grid_for(total, 256), 256, 0, st>>>(g, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t launch_init_spins(const Group &g, uint64_t seed, cudaStream_t st) {
    count_launches(1);
    k_init_spins<<<grid_for((long long)g.nslots * g.N, 256), 256, 0, st>>>(g, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t launch_sweep_reference(const Group &g, uint32_t sweep, uint64_t seed, cudaStream_t st) {
    const long long work = (long long)g.N / 2 * g.nslots;
    for (int colour = 0; colour < 2; ++colour) {
        count_launches(1);
        k_half_sweep_ref<<<grid_for(work, 256), 256, 0, st>>>(g, colour, sweep, (uint32_t)seed, (uint32_t)(seed >> 32));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qsg
