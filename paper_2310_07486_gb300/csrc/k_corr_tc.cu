// k_corr_tc.cu -- imaginary-time correlators on the 5th-generation tensor cores.
//
// For one sample (one bit of one slot) the correlators of Eq. (def-C-Q2-tau)
// are sums along the cyclic diagonals of the Gram matrix of its tau slices,
//     G(t1, t2) = sum_x S_x,t1 S_x,t2,
//     C(d) = sum_t1 s G(t1, t1 + d),   Q(d) = sum_t1 G(t1, t1 + d)^2,
// a dense contraction over the L^2 sites.  The spins are +-1, exact in FP8
// E4M3, and every partial sum is an integer of magnitude <= L^2 < 2^24, so a
// tcgen05.mma (kind::f8f6f4, FP32 accumulation in tensor memory) computes G
// exactly.  Each CTA owns one 128-row block i of one sample and walks the
// column blocks j >= i (the upper triangle; G is symmetric), folding every
// element into per-lag bins: pairs with offset o = t2 - t1 feed lag o when
// o < L_tau/2 and lag L_tau - o (the forward pair from t2, which wraps, so it
// carries the APBC sign) when o > L_tau/2; o = L_tau/2 counts twice.
//
// Operands: the x-packed bit planes of the transposed scratch buffer are
// expanded to E4M3 +-1 (0 for padding) in shared memory, K-major with the
// 128-byte swizzle, in chunks of 128 sites, double buffered against the MMA.
#include "qsg_launch.h"

namespace qsg {

namespace {

constexpr int kTile = 128;          // rows of A (t1) and of B (t2) per tile
constexpr int kChunk = 128;         // sites (bytes) per K chunk = one swizzled row
constexpr int kChunkBytes = kTile * kChunk;  // 16 KB per operand chunk
constexpr int kThreads = 128;
constexpr unsigned kSpinLimit = 1u << 22;    // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D = FP32, A = B = E4M3, both K-major, M = N = 128.
__device__ __forceinline__ uint32_t idesc_e4m3_128x128() {
    return (1u << 4) | ((uint32_t)(kTile >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    uint32_t done = 0;
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(phase)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// 8 bits -> 8 bytes with 0x80 in the bytes whose bit is set
__device__ __forceinline__ uint64_t spread8(const uint64_t *lut, uint32_t bits) { return lut[bits & 0xFF]; }

}  // namespace

// grid: (row blocks nb, slots-bits of the batch); P: [slot_b][bit][Ltau][nwx]
__global__ void __launch_bounds__(kThreads) k_gram_tc(Group g, int p0, const uint64_t *__restrict__ P, int nb,
                                                      int *status) {
    extern __shared__ __align__(16) uint8_t dyn_raw[];
    // the 128-byte swizzle wants 1024-byte aligned operand chunks
    uint8_t *dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);
    uint8_t *sbuf = dyn;                                   // [2 buffers][A, B][16 KB]
    uint64_t *lut = reinterpret_cast<uint64_t *>(dyn + 4 * kChunkBytes);   // 256 entries
    int *binC = reinterpret_cast<int *>(lut + 256);        // [nlag]
    int *binQ = binC + g.nlag;                             // [nlag]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i = blockIdx.x;                 // row block
    const int sbb = blockIdx.y;               // (slot of batch, bit)
    const int sb = sbb / 64, bit = sbb % 64;
    const int pb = sb / g.R, r = sb % g.R;
    const int pidx = p0 + pb, w = pidx / g.K, j = pidx % g.K;
    const int Lt = g.Ltau, nwx = g.nwx, L2 = g.L * g.L, half = Lt / 2;
    const int nchunks = (L2 + kChunk - 1) / kChunk;
    const uint64_t *src = P + ((size_t)sb * 64 + bit) * Lt * nwx;

    for (int v = tid; v < 256; v += kThreads) {
        uint64_t x = 0;
        for (int q = 0; q < 8; ++q)
            if (v >> q & 1) x |= 0x80ull << (8 * q);
        lut[v] = x;
    }
    for (int l = tid; l < g.nlag; l += kThreads) binC[l] = binQ[l] = 0;
    if (tid == 0) abort_flag = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_e4m3_128x128();

    // expand rows [blk*128, blk*128+128) of K chunk kc into a swizzled operand chunk
    auto expand = [&](uint8_t *dst, int blk, int kc) {
        const int row = tid;                      // one row per thread
        const int t = blk * kTile + row;
        const int k0 = kc * kChunk;
        uint64_t wlo = 0, whi = 0;
        int valid = 0;
        if (t < Lt) {
            const int w0 = k0 / 64;
            wlo = w0 < nwx ? src[(size_t)t * nwx + w0] : 0ull;
            whi = w0 + 1 < nwx ? src[(size_t)t * nwx + w0 + 1] : 0ull;
            valid = min(max(L2 - k0, 0), kChunk);
        }
        uint8_t *rowp = dst + row * 128;
#pragma unroll
        for (int c16 = 0; c16 < 8; ++c16) {
            const uint64_t wsrc = c16 < 4 ? wlo : whi;
            const int sh = (c16 & 3) * 16;
            const uint32_t b16 = (uint32_t)(wsrc >> sh) & 0xFFFFu;
            // validity of the 16 sites of this 16-byte chunk
            const int nv = min(max(valid - c16 * 16, 0), 16);
            const uint32_t v16 = nv >= 16 ? 0xFFFFu : ((1u << nv) - 1u);
            const uint64_t lo = (spread8(lut, b16) | 0x3838383838383838ull) & ((spread8(lut, v16) >> 7) * 0xFFull);
            const uint64_t hi = (spread8(lut, b16 >> 8) | 0x3838383838383838ull) & ((spread8(lut, v16 >> 8) >> 7) * 0xFFull);
            *reinterpret_cast<ulonglong2 *>(rowp + ((c16 ^ (row & 7)) << 4)) = make_ulonglong2(lo, hi);
        }
    };

    uint32_t phase[2] = {0, 0};
    int issued[2] = {0, 0};   // commits outstanding per buffer
    int gchunk = 0;           // running chunk index (buffer = gchunk & 1)
    bool ok = true;

    for (int jb = i; jb < nb && ok; ++jb) {
        for (int kc = 0; kc < nchunks; ++kc, ++gchunk) {
            const int buf = gchunk & 1;
            // the MMA that last read this buffer must be complete; every thread
            // waits and the block agrees on the outcome before going on
            bool mine = true;
            if (issued[buf]) {
                mine = mbar_wait(smem_u32(&mbar[buf]), phase[buf]);
                phase[buf] ^= 1u;
                issued[buf] = 0;
            }
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
            uint8_t *sA = sbuf + buf * 2 * kChunkBytes, *sB = sA + kChunkBytes;
            expand(sA, i, kc);
            expand(sB, jb, kc);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
                for (int kk = 0; kk < kChunk / 32; ++kk) {
                    const uint64_t da = sdesc_sw128(smem_u32(sA) + kk * 32);
                    const uint64_t db = sdesc_sw128(smem_u32(sB) + kk * 32);
                    const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&mbar[buf])));
            }
            issued[buf] = 1;
        }
        if (!ok) break;
        // wait for the tile's last MMA, then fold the accumulator into the lag bins
        const int lastbuf = (gchunk - 1) & 1;
        const bool mine = mbar_wait(smem_u32(&mbar[lastbuf]), phase[lastbuf]);
        phase[lastbuf] ^= 1u;
        issued[lastbuf] = 0;
        ok = __syncthreads_and(mine) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const int m = warp * 32 + lane;       // TMEM lane = row of the tile
        const int t1 = i * kTile + m;
#pragma unroll 1
        for (int c0 = 0; c0 < kTile; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (t1 < Lt) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int t2 = jb * kTile + c0 + q;
                    const int o = t2 - t1;
                    if (t2 < Lt && o > 0) {
                        const int gv = __float2int_rn(__uint_as_float(v[q]));
                        int lag, wc, wq;
                        if (o < half) {
                            lag = o; wc = 1; wq = 1;
                        } else if (o == half) {
                            lag = half; wc = g.boundary == 1 ? 0 : 2; wq = 2;
                        } else {
                            lag = Lt - o; wc = g.boundary == 1 ? -1 : 1; wq = 1;
                        }
                        atomicAdd(&binC[lag], wc * gv);
                        atomicAdd(&binQ[lag], wq * gv * gv);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();   // the next tile's first MMA overwrites the accumulator
    }
    if (!ok && tid == 0) atomicExch(&abort_flag, 1);
    // drain: make sure no MMA is still reading shared memory or writing TMEM
    for (int b = 0; b < 2; ++b)
        if (issued[b]) mbar_wait(smem_u32(&mbar[b]), phase[b]);
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
    if (abort_flag) {
        if (tid == 0) atomicExch(status, DEVERR_TIMEOUT);
        return;
    }
    // the diagonal (lag 0) is G(t, t) = L^2 for every t: added once per sample
    const size_t base = ((((size_t)r * g.W * 64) + (size_t)w * 64 + bit) * g.K + j) * g.nlag;
    for (int l = tid; l < g.nlag; l += kThreads) {
        long long c = binC[l], q = binQ[l];
        if (l == 0 && i == 0) {
            c += (long long)Lt * L2;
            q += (long long)Lt * L2 * L2;
        }
        if (c) atomicAdd(reinterpret_cast<unsigned long long *>(&g.Cacc[base + l]), (unsigned long long)c);
        if (q) atomicAdd(reinterpret_cast<unsigned long long *>(&g.Qacc[base + l]), (unsigned long long)q);
    }
}

size_t gram_tc_smem_bytes(const Group &g) {
    return 1024 + 4 * (size_t)kChunkBytes + 256 * sizeof(uint64_t) + 2 * sizeof(int) * (size_t)g.nlag;
}

cudaError_t launch_gram_tc(const Group &g, int p0, int npairs, const uint64_t *P, int *status, cudaStream_t st) {
    const int nb = (g.Ltau + kTile - 1) / kTile;
    const size_t sm = gram_tc_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(nb, npairs * g.R * 64);
    count_launches(1);
    k_gram_tc<<<grid, kThreads, sm, st>>>(g, p0, P, nb, status);
    return cudaGetLastError();
}

}  // namespace qsg
