// k_corr.cu -- imaginary-time correlators C(tau), Q2(tau) and the equal-time
// replica overlap (Eqs. (C_A_transfer), (def-C-Q2-tau)), accumulated exactly
// in int64, and their FP64 finish.
//
// The multispin words hold 64 samples per site.  The correlators need, per
// sample, the overlap of two tau slices summed over sites, so the slices are
// first transposed into x-packed words (64 sites per word, one sample per
// row) in a scratch buffer; an overlap is then L^2 - 2 popc(a ^ b).
#include "qsg_launch.h"

namespace qsg {

size_t measure_scratch_words_per_pair(const Group &g) {
    return (size_t)g.R * 64 * g.Ltau * g.nwx;
}

// Bit matrix transpose step of half-size j across lanes l and l ^ j: bits
// whose index has bit j clear (mask m) stay in the lower row; the lower row
// takes the partner's low-half bits shifted up, the upper row the partner's
// high-half bits shifted down.  Five such steps (j = 16 .. 1) and the
// in-register step j = 32 swap the bits of (row, column): (s, b) -> (b, s).
template <int J>
__device__ __forceinline__ uint64_t transpose_step(uint64_t w, bool upper, uint64_t m) {
    const uint64_t p = __shfl_xor_sync(0xffffffffu, w, J);
    return upper ? ((w & ~m) | ((p >> J) & m)) : ((w & m) | ((p << J) & ~m));
}

// scratch layout for a batch of (w, j) pairs: [pair][r][b][tau][nwx].
// One block per (slot of the batch, run of kTrRun tau planes), one warp per
// plane: for every 64-site group the warp's lane l loads the multispin words
// of sites l and l + 32 (bit b = sample b, one coalesced 512-byte read),
// transposes the 64 x 64 bit block in registers and holds the x-packed words
// of samples l and l + 32, which it puts in shared memory.  The block then
// writes each sample's kTrRun x nwx words, contiguous in the scratch, as one
// coalesced run (a sample's words of one plane are nwx words long and the
// next sample's begin L_tau nwx words later, so a warp storing its two words
// straight would write 64 separate 8-byte pieces).
constexpr int kTrRun = 8;  // tau planes per block (warps of 32 threads)

__global__ void __launch_bounds__(32 * kTrRun) k_transpose(Group g, int p0, int npairs, uint64_t *P) {
    extern __shared__ uint64_t trs[];  // [64 samples][kTrRun * nwx + 1 (padding)]
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int nwx = g.nwx, Lt = g.Ltau, L2 = g.L * g.L;
    const int pitch = kTrRun * nwx + 1;
    const int sb = blockIdx.x;  // slot of the batch: (pair, replica)
    const int t0 = blockIdx.y * kTrRun, nt = min(kTrRun, Lt - t0);
    const int pb = sb / g.R, r = sb % g.R;
    const int p = p0 + pb, w = p / g.K, j = p % g.K;
    const size_t s = ((size_t)w * g.R + r) * g.K + j;
    if (sb >= npairs * g.R) return;  // the grid is exact: never taken
    if (wp < nt) {
        const int t = t0 + wp;
        const uint64_t *src = g.S + s * g.N + (size_t)t * L2;
        for (int gx = 0; gx < nwx; ++gx) {
            const int s0 = gx * 64 + lane, s1 = s0 + 32;
            const uint64_t w0 = s0 < L2 ? src[s0] : 0ull;
            const uint64_t w1 = s1 < L2 ? src[s1] : 0ull;
            // j = 32: rows l and l + 32 are both in this lane
            uint64_t a0 = (w0 & 0xFFFFFFFFull) | (w1 << 32);
            uint64_t a1 = (w0 >> 32) | (w1 & 0xFFFFFFFF00000000ull);
            a0 = transpose_step<16>(a0, lane & 16, 0x0000FFFF0000FFFFull);
            a1 = transpose_step<16>(a1, lane & 16, 0x0000FFFF0000FFFFull);
            a0 = transpose_step<8>(a0, lane & 8, 0x00FF00FF00FF00FFull);
            a1 = transpose_step<8>(a1, lane & 8, 0x00FF00FF00FF00FFull);
            a0 = transpose_step<4>(a0, lane & 4, 0x0F0F0F0F0F0F0F0Full);
            a1 = transpose_step<4>(a1, lane & 4, 0x0F0F0F0F0F0F0F0Full);
            a0 = transpose_step<2>(a0, lane & 2, 0x3333333333333333ull);
            a1 = transpose_step<2>(a1, lane & 2, 0x3333333333333333ull);
            a0 = transpose_step<1>(a0, lane & 1, 0x5555555555555555ull);
            a1 = transpose_step<1>(a1, lane & 1, 0x5555555555555555ull);
            trs[(size_t)lane * pitch + wp * nwx + gx] = a0;
            trs[(size_t)(lane + 32) * pitch + wp * nwx + gx] = a1;
        }
    }
    __syncthreads();
    // sample b's words of planes t0 .. t0 + nt - 1 are contiguous in the scratch
    const int n = nt * nwx;
    uint64_t *dst = P + ((size_t)sb * 64 * Lt + t0) * nwx;
    for (int b = wp; b < 64; b += kTrRun)
        for (int o = lane; o < n; o += 32) dst[(size_t)b * Lt * nwx + o] = trs[(size_t)b * pitch + o];
}

// One block per (slot of the batch, sample bit): all lags of one sample.
__global__ void __launch_bounds__(256) k_gram(Group g, int p0, const uint64_t *P, int use_smem) {
    extern __shared__ uint64_t sh[];
    const int sb = blockIdx.x / 64, b = blockIdx.x % 64;
    const int pb = sb / g.R, r = sb % g.R;
    const int p = p0 + pb, w = p / g.K, j = p % g.K;
    const int Lt = g.Ltau, nwx = g.nwx, L2 = g.L * g.L;
    const uint64_t *src = P + ((size_t)sb * 64 + b) * Lt * nwx;
    if (use_smem) {
        for (int i = threadIdx.x; i < Lt * nwx; i += blockDim.x) sh[i] = src[i];
        __syncthreads();
        src = sh;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int lag = warp; lag < g.nlag; lag += nwarp) {
        long long cs = 0, qs = 0;
        for (int t1 = lane; t1 < Lt; t1 += 32) {
            int t2 = t1 + lag;
            int sgn = 1;
            if (t2 >= Lt) {
                t2 -= Lt;
                if (g.boundary == 1) sgn = -1;
            }
            int d = 0;
            for (int x = 0; x < nwx; ++x) d += __popcll(src[t1 * nwx + x] ^ src[t2 * nwx + x]);
            const long long c = (long long)(L2 - 2 * d);
            cs += sgn * c;
            qs += c * c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cs += __shfl_down_sync(0xffffffffu, cs, o);
            qs += __shfl_down_sync(0xffffffffu, qs, o);
        }
        if (lane == 0) {
            const size_t idx = ((((size_t)r * g.W * 64) + (size_t)w * 64 + b) * g.K + j) * g.nlag + lag;
            g.Cacc[idx] += cs;
            g.Qacc[idx] += qs;
        }
    }
}

// Equal-time overlap of every replica pair at one ladder position.
cudaError_t launch_measure(const Group &g, uint64_t *scratch, size_t scratch_words, int tensor, int triples,
                           int *status, unsigned wait_limit, cudaStream_t st) {
    if (tensor && !gram_tc_fits(g)) tensor = 0;  // very long L_tau: integer pipes
    const size_t per_pair = measure_scratch_words_per_pair(g);
    int batch = (int)(scratch_words / per_pair);
    if (batch < 1) return cudaErrorInvalidValue;
    const int npairs_total = g.W * g.K;
    const size_t sh_bytes = (size_t)g.Ltau * g.nwx * sizeof(uint64_t);
    const int use_smem = sh_bytes <= 200 * 1024 ? 1 : 0;
    if (use_smem && !tensor) {
        cudaError_t e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_bytes);
        if (e != cudaSuccess) return e;
    }
    for (int p0 = 0; p0 < npairs_total; p0 += batch) {
        const int np = min(batch, npairs_total - p0);
        const size_t tr_smem = (size_t)64 * (kTrRun * g.nwx + 1) * sizeof(uint64_t);
        if (tr_smem > 48 * 1024) {
            const cudaError_t ea = cudaFuncSetAttribute(k_transpose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)tr_smem);
            if (ea != cudaSuccess) return ea;
        }
        count_launches(1);
        // slots along x (up to 2^31 - 1), runs of planes along y (L_tau / 8 <= 8192)
        k_transpose<<<dim3((unsigned)(np * g.R), (unsigned)((g.Ltau + kTrRun - 1) / kTrRun)), 32 * kTrRun, tr_smem,
                      st>>>(g, p0, np, scratch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (tensor) {
            e = launch_gram_tc(g, p0, np, scratch, status, wait_limit, st);
        } else {
            count_launches(1);
            k_gram<<<np * g.R * 64, 256, use_smem ? sh_bytes : 0, st>>>(g, p0, scratch, use_smem);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
        // equal-time replica overlaps and the other one-time sums (k_onetime.cu)
        e = launch_onetime(g, p0, np, scratch, triples, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// C = C_acc / (n_meas L^2 L_tau), Q2 = Q_acc / (n_meas L^4 L_tau),
// q2 = P_acc / (n_meas n_pairs L^4 L_tau); IEEE division, no fused operations.
__global__ void k_finish(Group g, double nm) {
    const double L2 = (double)(g.L * g.L), Lt = (double)g.Ltau;
    const double pairs = (double)(g.R * (g.R - 1) / 2);
    const size_t nc = (size_t)g.R * g.W * 64 * g.K * g.nlag;
    const size_t np = (size_t)g.W * 64 * g.K;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nc; i += (size_t)gridDim.x * blockDim.x) {
        g.outC[i] = __ddiv_rn((double)g.Cacc[i], __dmul_rn(__dmul_rn(nm, L2), Lt));
        g.outQ[i] = __ddiv_rn((double)g.Qacc[i], __dmul_rn(__dmul_rn(__dmul_rn(nm, L2), L2), Lt));
        if (i < np)
            g.outP[i] = __ddiv_rn((double)g.Pacc[i],
                                  __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(nm, pairs), L2), L2), Lt));
    }
}

cudaError_t launch_finish(const Group &g, long long n_meas, cudaStream_t st) {
    const size_t nc = (size_t)g.R * g.W * 64 * g.K * g.nlag;
    long long blocks = (long long)((nc + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_launches(1);
    k_finish<<<(int)blocks, 256, 0, st>>>(g, (double)n_meas);
    return cudaGetLastError();
}

}  // namespace qsg
