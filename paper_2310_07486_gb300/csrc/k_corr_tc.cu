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
// 128-byte swizzle, in chunks of 128 sites, double buffered against the MMA;
// four spin bits become four bytes with one multiply and one mask.
#include "qsg_launch.h"

namespace qsg {

namespace {

constexpr int kTile = 128;          // rows of A (t1) and of B (t2) per tile
constexpr int kChunk = 128;         // sites (bytes) per K chunk = one swizzled row
constexpr int kChunkBytes = kTile * kChunk;  // 16 KB per operand chunk
constexpr int kThreads = 256;  // two threads per tile row (expansion), two warps per TMEM lane quadrant
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

}  // namespace

// 4 spin bits -> 4 E4M3 bytes: +1 = 0x38, -1 = 0xB8 (a set bit is spin -1).
// The multiplier places bit k at bit 8k + 7; the four shifted copies of the
// nibble do not overlap, so no carry disturbs the kept bits.
__device__ __forceinline__ uint32_t nibble_e4m3(uint32_t x4) {
    return ((x4 * 0x10204080u) & 0x80808080u) | 0x38383838u;
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// grid: (row blocks nb, slot-bits of the batch); P: [slot_b][bit][Ltau][nwx].
// Shared memory: operand chunks [2 buffers][A, B][16 KB] (1024-aligned), the
// lag bins, and the bit rows of the A block and of two B blocks (the next one
// is fetched while the current one is multiplied).
__global__ void __launch_bounds__(kThreads) k_gram_tc(Group g, int p0, const uint64_t *__restrict__ P, int nb,
                                                      int *status) {
    extern __shared__ __align__(16) uint8_t dyn_raw[];
    uint8_t *dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);
    const int Lt = g.Ltau, nwx = g.nwx, L2 = g.L * g.L, half = Lt / 2;
    uint8_t *sbuf = dyn;
    int *binC = reinterpret_cast<int *>(dyn + 4 * kChunkBytes);
    int *binQ = binC + g.nlag;
    uint64_t *bitsA = reinterpret_cast<uint64_t *>(binQ + g.nlag);
    bitsA = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(bitsA) + 15) & ~(uintptr_t)15);
    uint64_t *bitsB = bitsA + kTile * nwx;  // [2][kTile][nwx]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i = blockIdx.x;
    const int sbb = blockIdx.y;
    const int sb = sbb / 64, bit = sbb % 64;
    const int pb = sb / g.R, r = sb % g.R;
    const int pidx = p0 + pb, w = pidx / g.K, j = pidx % g.K;
    const int nchunks = (L2 + kChunk - 1) / kChunk;
    const uint64_t *src = P + ((size_t)sb * 64 + bit) * Lt * nwx;

    // bit rows of block blk into dst (threads < 128, one row each; rows past L_tau are zero)
    auto fetch_rows = [&](uint64_t *dst, int blk) {
        if (tid < kTile) {
            const int t = blk * kTile + tid;
            uint64_t *d = dst + tid * nwx;
            if (t < Lt) {
                for (int x = 0; x < nwx; ++x) cp_async8(d + x, src + (size_t)t * nwx + x);
            } else {
                for (int x = 0; x < nwx; ++x) d[x] = 0ull;
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    fetch_rows(bitsA, i);
    fetch_rows(bitsB, i);
    for (int l = tid; l < g.nlag; l += kThreads) binC[l] = binQ[l] = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_e4m3_128x128();

    // expand K chunk kc of the bit rows `bits` into a swizzled E4M3 operand
    // chunk; thread = (row, half row of 64 sites = one bit word)
    auto expand = [&](uint8_t *dst, const uint64_t *bits, int blk, int kc) {
        const int row = tid >> 1, hh = tid & 1;
        const int t = blk * kTile + row;
        const int k0 = kc * kChunk + 64 * hh;
        const int wi = k0 / 64;
        const uint64_t word = wi < nwx ? bits[row * nwx + wi] : 0ull;
        const int valid = t < Lt ? min(max(L2 - k0, 0), 64) : 0;
        uint8_t *rowp = dst + row * 128;
        // E4M3: +1 = 0x38, -1 = 0xB8 (set bit = spin -1), 0 for padding sites
#pragma unroll
        for (int gq = 0; gq < 4; ++gq) {
            const uint32_t b16 = (uint32_t)(word >> (gq * 16));
            uint32_t out[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) out[qq] = nibble_e4m3((b16 >> (4 * qq)) & 0xFu);
            if (valid < 64) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
#pragma unroll
                    for (int by = 0; by < 4; ++by)
                        if (gq * 16 + qq * 4 + by >= valid) out[qq] &= ~(0xFFu << (8 * by));
            }
            *reinterpret_cast<uint4 *>(rowp + (((4 * hh + gq) ^ (row & 7)) << 4)) =
                make_uint4(out[0], out[1], out[2], out[3]);
        }
    };

    uint32_t phase[2] = {0, 0};
    int issued[2] = {0, 0};
    int gchunk = 0;
    bool ok = true;
    // epilogue: warp -> TMEM lane quadrant (rows) and one half of the columns
    const int m = (warp & 3) * 32 + lane;  // TMEM lane = tile row
    const int cbase = (warp >> 2) * 64;
    const int t1 = i * kTile + m;

    for (int jb = i; jb < nb && ok; ++jb) {
        const uint64_t *bb = bitsB + (size_t)((jb - i) & 1) * kTile * nwx;
        // fetch the next B block while this one is multiplied
        if (jb + 1 < nb) fetch_rows(bitsB + (size_t)((jb + 1 - i) & 1) * kTile * nwx, jb + 1);
        for (int kc = 0; kc < nchunks; ++kc, ++gchunk) {
            const int buf = gchunk & 1;
            bool mine = true;
            if (issued[buf]) {
                mine = mbar_wait(smem_u32(&mbar[buf]), phase[buf]);
                phase[buf] ^= 1u;
                issued[buf] = 0;
            }
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
            uint8_t *sA = sbuf + buf * 2 * kChunkBytes, *sB = sA + kChunkBytes;
            expand(sA, bitsA, i, kc);
            expand(sB, bb, jb, kc);
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
        const int lastbuf = (gchunk - 1) & 1;
        const bool mine = mbar_wait(smem_u32(&mbar[lastbuf]), phase[lastbuf]);
        phase[lastbuf] ^= 1u;
        issued[lastbuf] = 0;
        ok = __syncthreads_and(mine) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        // offsets o = t2 - t1 of this tile lie in [omin, omax]; most tiles map
        // every element to lag o (all o < L_tau/2) or to lag L_tau - o (all o >
        // L_tau/2), only the tiles around L_tau/2 need the per-element choice
        const int obase = (jb - i) * kTile;
        const int omin = jb == i ? 1 : obase - (kTile - 1), omax = obase + kTile - 1;
        const bool full = (jb + 1) * kTile <= Lt && (i + 1) * kTile <= Lt;
        const int cls = (omax < half) ? 0 : (omin > half ? 1 : 2);
        const int whigh = g.boundary == 1 ? -1 : 1;
#pragma unroll 1
        for (int c0 = cbase; c0 < cbase + 64; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            const int o0 = obase + c0 - m;  // offset of column q is o0 + q
            if (full && cls == 0 && jb != i) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int gv = __float2int_rn(__uint_as_float(v[q]));
                    atomicAdd(&binC[o0 + q], gv);
                    atomicAdd(&binQ[o0 + q], gv * gv);
                }
            } else if (full && cls == 1) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int gv = __float2int_rn(__uint_as_float(v[q]));
                    atomicAdd(&binC[Lt - o0 - q], whigh * gv);
                    atomicAdd(&binQ[Lt - o0 - q], gv * gv);
                }
            } else if (t1 < Lt) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int t2 = jb * kTile + c0 + q;
                    const int o = o0 + q;
                    if (t2 < Lt && o > 0) {
                        const int gv = __float2int_rn(__uint_as_float(v[q]));
                        int lag, wc, wq;
                        if (o < half) {
                            lag = o; wc = 1; wq = 1;
                        } else if (o == half) {
                            lag = half; wc = g.boundary == 1 ? 0 : 2; wq = 2;
                        } else {
                            lag = Lt - o; wc = whigh; wq = 1;
                        }
                        atomicAdd(&binC[lag], wc * gv);
                        atomicAdd(&binQ[lag], wq * gv * gv);
                    }
                }
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();  // next B rows visible; the next tile may overwrite the accumulator
    }
    const bool failed = !ok;
    for (int b = 0; b < 2; ++b)
        if (issued[b]) mbar_wait(smem_u32(&mbar[b]), phase[b]);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
    if (failed) {
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
    return 1024 + 4 * (size_t)kChunkBytes + 2 * sizeof(int) * (size_t)g.nlag + 16 +
           3 * (size_t)kTile * g.nwx * sizeof(uint64_t);
}

bool gram_tc_fits(const Group &g) { return gram_tc_smem_bytes(g) <= 227 * 1024; }

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
