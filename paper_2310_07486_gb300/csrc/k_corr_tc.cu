// k_corr_tc.cu -- imaginary-time correlators on the 5th-generation tensor cores.
//
// For one sample (one bit of one slot) the correlators of Eq. (def-C-Q2-tau)
// are sums along the cyclic diagonals of the Gram matrix of its tau slices,
//     G(t1, t2) = sum_x S_x,t1 S_x,t2,
//     C(d) = sum_t1 s G(t1, t1 + d),   Q(d) = sum_t1 G(t1, t1 + d)^2,
// a dense contraction over the L^2 sites.  The spins are +-1, exact in FP8
// E4M3, and every partial sum is an integer of magnitude <= L^2 < 2^24, so a
// tcgen05.mma (kind::f8f6f4, FP32 accumulation in tensor memory) computes G
// exactly.  Only the upper triangle of 128 x 128 tiles (i, j >= i) is formed
// (G is symmetric), and every element is folded into per-lag bins: pairs with
// offset o = t2 - t1 feed lag o when o < L_tau/2 and lag L_tau - o (the
// forward pair from t2, which wraps, so it carries the APBC sign) when
// o > L_tau/2; o = L_tau/2 counts twice.
//
// One persistent CTA per SM, specialised warps:
//   producers (8 warps, two threads per tile row) load the x-packed bit rows
//     of the transposed scratch one row block ahead into registers and expand
//     them to E4M3 +-1 (0 for padding) in shared memory, K-major with the
//     128-byte swizzle, sites in a bit-interleaved order shared by A and B:
//     the A row block once (resident, double buffered where shared memory
//     allows, while its row of tiles is multiplied), B in 128-site chunks
//     through a ring of stages;
//   one thread issues the MMAs into two tensor-memory accumulators, so the
//     next tile is multiplied while the last one is folded;
//   the epilogue (8 warps, two per TMEM lane quadrant) folds the tiles into
//     shared-memory lag bins and flushes them to the int64 sums.
// The work unit is one sample's row blocks i and nb - 1 - i: nb + 1 tiles for
// every unit, so a static round robin over the units balances the SMs.
#include "qsg_launch.h"

namespace qsg {

namespace {

constexpr int kTile = 128;                   // rows of A (t1) and of B (t2) per tile
constexpr int kChunk = 128;                  // sites (bytes) per K chunk = one swizzled row
constexpr int kChunkBytes = kTile * kChunk;  // 16 KB per operand chunk
constexpr int kMaxNc = 8;                    // 128-site chunks of a row at most (L <= 32)
constexpr int kMaxStages = 6;                // B stages at most
constexpr int kProducers = 256;              // warps 0-7: two threads per tile row
constexpr int kProducerWarps = kProducers / 32;
constexpr int kEpilogueWarps = 8;
constexpr int kEpilogue = 256;               // warps 8-15: two per TMEM lane quadrant
constexpr int kMmaWarp = 16;
constexpr int kThreads = 17 * 32;
constexpr unsigned kSpinLimit = 1u << 22;    // polls of the wait for issued MMAs before TMEM is freed

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

struct Ctl {
    uint64_t bfull[kMaxStages], bempty[kMaxStages];  // B stage written / multiplied
    uint64_t afull[2], aempty[2];                    // A buffer written / multiplied
    uint64_t accfull[2], accempty[2];                // accumulator computed / folded
    uint64_t done;                                   // every MMA of the CTA completed
    uint32_t tmem;
    int abort;  // a wait gave up: every role skips its work and runs out its loops
};

// Wait for the phase of the given parity; false (and the abort flag set) when
// `limit` polls are used up or another thread has given up already.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *abort, unsigned limit) {
    volatile int *ab = abort;
    if (*ab) return false;
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && *ab) return false;
    }
    *ab = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 spin bits -> 32 E4M3 bytes (+1 = 0x38, -1 = 0xB8; a set bit is spin -1)
// in the site order of the contraction: byte k of output word j is bit
// 8k + j.  The Gram sums over sites, so any order serves that A and B share;
// this one takes one shift and one mask per output word.
__device__ __forceinline__ uint32_t spread_e4m3(uint32_t b, int j) {
    return ((b << (7 - j)) & 0x80808080u) | 0x38383838u;
}

// Bytes of spread_e4m3's output word j whose bits are set in the site mask vm
// are 0xFF, the others 0.
__device__ __forceinline__ uint32_t spread_mask(uint32_t vm, int j) {
    return (((vm << (7 - j)) & 0x80808080u) >> 7) * 0xFFu;
}

// The 64 sites of word wv into granules 4 hh .. 4 hh + 3 of the swizzled
// 128-byte row `row` at rowp; sites >= valid (outside the lattice, or every
// site of a row past L_tau) become 0.  Output words 8 e + j (e = half of the
// word) fill granules 4 hh + 2 e + (j >> 2).
__device__ __forceinline__ void expand_full(uint8_t *rowp, uint64_t wv, int hh, int row) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const uint32_t b = (uint32_t)(wv >> (32 * e));
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
            const int gr = 4 * hh + 2 * e + hq;
            *reinterpret_cast<uint4 *>(rowp + ((gr ^ (row & 7)) << 4)) =
                make_uint4(spread_e4m3(b, 4 * hq), spread_e4m3(b, 4 * hq + 1), spread_e4m3(b, 4 * hq + 2),
                           spread_e4m3(b, 4 * hq + 3));
        }
    }
}

__device__ __noinline__ void expand_part(uint8_t *rowp, uint64_t wv, int valid, int hh, int row) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const uint32_t b = (uint32_t)(wv >> (32 * e));
        const int v32 = valid - 32 * e;
        const uint32_t vm = v32 >= 32 ? 0xFFFFFFFFu : (v32 <= 0 ? 0u : (1u << v32) - 1u);
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
            const int gr = 4 * hh + 2 * e + hq;
            uint32_t o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = spread_e4m3(b, 4 * hq + k) & spread_mask(vm, 4 * hq + k);
            *reinterpret_cast<uint4 *>(rowp + ((gr ^ (row & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

__device__ __forceinline__ void expand_word(uint8_t *rowp, uint64_t wv, int valid, int hh, int row) {
    if (valid >= 64)
        expand_full(rowp, wv, hh, row);
    else
        expand_part(rowp, wv, valid, hh, row);
}

// The work of one CTA: units u = blockIdx.x + n gridDim.x; unit u is sample
// u / nhalf, row blocks h = u % nhalf and nb - 1 - h (one block when equal).
// Within a unit the blocks are items; item i has the tiles (i, jb), jb >= i.
// The producers' block sequence per item: the A block i, then the B blocks
// jb = i+1..nb-1 (tile (i, i) takes B = A).
struct Blk {
    int u, sidx, h, item, i, jb;
    bool valid;
};

__device__ __forceinline__ int item_block(int h, int item, int nb) { return item ? nb - 1 - h : h; }
__device__ __forceinline__ int unit_items(int h, int nb) { return nb - 1 - h != h ? 2 : 1; }

__device__ __forceinline__ void blk_unit(Blk &c, int nunits, int nhalf) {
    c.valid = c.u < nunits;
    c.sidx = c.u / nhalf;
    c.h = c.u - c.sidx * nhalf;
    c.item = 0;
    c.i = c.h;
    c.jb = c.h;
}

__device__ __forceinline__ void blk_first(Blk &c, int nunits, int nhalf) {
    c.u = blockIdx.x;
    blk_unit(c, nunits, nhalf);
}

__device__ __forceinline__ void blk_next(Blk &c, int nunits, int nhalf, int nb) {
    if (++c.jb < nb) return;
    if (++c.item >= unit_items(c.h, nb)) {
        c.u += gridDim.x;
        blk_unit(c, nunits, nhalf);
        return;
    }
    c.i = item_block(c.h, c.item, nb);
    c.jb = c.i;
}

// Bit words of thread (row, hh) in a block: w[kc] = word 2 kc + hh of row
// jb * 128 + row, 0 outside the lattice and past L_tau.
__device__ __forceinline__ void load_blk(const Blk &c, const uint64_t *__restrict__ P, int Lt, int nwx, int nc, int row,
                                         int hh, uint64_t (&w)[kMaxNc]) {
    const int t = c.jb * kTile + row;
    const bool in = c.valid && t < Lt;
    const uint64_t *src = P + ((size_t)(c.valid ? c.sidx : 0) * Lt + (t < Lt ? t : 0)) * nwx + hh;
#pragma unroll
    for (int kc = 0; kc < kMaxNc; ++kc)
        if (kc < nc) w[kc] = (in && 2 * kc + hh < nwx) ? __ldg(src + 2 * kc) : 0ull;
}

// FP32 accumulator holding an integer |x| < 2^22 -> int32 with one add: in
// [2^23, 2^24) the FP32 spacing is 1, so x + 1.5 * 2^23 is exact and its bit
// pattern is that of 1.5 * 2^23 plus x.
__device__ __forceinline__ int exact_f32_to_int(uint32_t bits) {
    return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

}  // namespace

// P: [sample][Ltau][nwx] transposed bits of the batch (sample = (pair, r, bit)).
__global__ void __launch_bounds__(kThreads, 1)
    k_gram_tc(Group g, int p0, const uint64_t *__restrict__ P, int nsamples, int nstages, int nabuf, int *status,
              unsigned wait_limit) {
    extern __shared__ __align__(16) uint8_t dyn_raw[];
    uint8_t *dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);
    __shared__ Ctl ctl;
    const int Lt = g.Ltau, L2 = g.L * g.L, half = Lt / 2, nl = g.nlag, nwx = g.nwx;
    const int nb = (Lt + kTile - 1) / kTile, nhalf = (nb + 1) / 2;
    const int nc = (L2 + kChunk - 1) / kChunk;
    const int nunits = nsamples * nhalf;
    uint8_t *sA = dyn;
    uint8_t *sB = sA + (size_t)nabuf * nc * kChunkBytes;  // A buffers, then the B stages
    int *binC = reinterpret_cast<int *>(sB + (size_t)nstages * kChunkBytes);
    unsigned *binQ = reinterpret_cast<unsigned *>(binC + nl);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&ctl.bfull[s])), "r"(kProducerWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&ctl.bempty[s])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&ctl.afull[b])), "r"(kProducerWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&ctl.aempty[b])));
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&ctl.accfull[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&ctl.accempty[a])), "r"(kEpilogueWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&ctl.done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        ctl.abort = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(smem_u32(&ctl.tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    for (int l = tid; l < nl; l += kThreads) {
        binC[l] = 0;
        binQ[l] = 0u;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = ctl.tmem;

    if (warp < kProducers / 32) {
        // ------------------------------------------------------------ producers
        // thread (row, hh): sites 64 hh .. 64 hh + 63 of every 128-site chunk of
        // a tile row; the bit words of the next block are loaded into registers
        // while the current block is expanded
        const int row = tid >> 1, hh = tid & 1;
        Blk cur, nxt;
        blk_first(cur, nunits, nhalf);
        uint64_t wc[kMaxNc], wn[kMaxNc];
        load_blk(cur, P, Lt, nwx, nc, row, hh, wc);
        // aempty / bempty[s] parities: the first use of a buffer waits for the
        // phase before the first (complete at initialisation)
        uint32_t a_par = 3u, b_par = 1u;  // a_par: bit b = parity of A buffer b
        int s = 0, ab = 0;
        while (cur.valid) {
            nxt = cur;
            blk_next(nxt, nunits, nhalf, nb);
            load_blk(nxt, P, Lt, nwx, nc, row, hh, wn);
            const int t = cur.jb * kTile + row;
            const bool isA = cur.jb == cur.i;  // the A block of an item
            uint8_t *abuf = sA + (size_t)ab * nc * kChunkBytes + row * kChunk;
#pragma unroll
            for (int kc = 0; kc < kMaxNc; ++kc) {
                if (kc < nc) {
                    bool ok = true;
                    if (!isA)
                        ok = mbar_wait(&ctl.bempty[s], b_par, &ctl.abort, wait_limit);
                    else if (kc == 0)
                        ok = mbar_wait(&ctl.aempty[ab], (a_par >> ab) & 1u, &ctl.abort, wait_limit);
                    uint8_t *rowp = isA ? abuf + (size_t)kc * kChunkBytes : sB + (size_t)s * kChunkBytes + row * kChunk;
                    if (ok) expand_word(rowp, wc[kc], t < Lt ? L2 - kc * kChunk - 64 * hh : 0, hh, row);
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    __syncwarp();  // the warp's rows are written: one arrival per warp
                    if (!isA) {
                        if (lane == 0) mbar_arrive(&ctl.bfull[s]);
                        if (++s == nstages) {
                            s = 0;
                            b_par ^= 1u;
                        }
                    } else if (kc == nc - 1) {
                        if (lane == 0) mbar_arrive(&ctl.afull[ab]);
                        a_par ^= 1u << ab;
                        if (++ab == nabuf) ab = 0;
                    }
                }
            }
#pragma unroll
            for (int kc = 0; kc < kMaxNc; ++kc) wc[kc] = wn[kc];
            cur = nxt;
        }
    } else if (warp < kMmaWarp) {
        // ------------------------------------------------------------- epilogue
        const int etid = tid - kProducers;
        const int quad = warp & 3;                       // TMEM lanes 32 quad .. 32 quad + 31
        const int cbase = ((warp - kProducers / 32) >> 2) * 64;  // column half of the tile
        const int m = quad * 32 + lane;                  // tile row
        const int whigh = g.boundary == 1 ? -1 : 1;
        uint32_t n_t = 0;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            const int sidx = u / nhalf, h = u % nhalf;
            for (int item = 0; item < unit_items(h, nb); ++item) {
                const int i = item_block(h, item, nb);
                const int t1 = i * kTile + m;
                for (int jb = i; jb < nb; ++jb, ++n_t) {
                    const int a = (int)(n_t & 1u);
                    const bool ok = mbar_wait(&ctl.accfull[a], (n_t >> 1) & 1u, &ctl.abort, wait_limit);
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    if (ok) {
                        // offsets o = t2 - t1 of this tile lie in [omin, omax]; most
                        // tiles map every element to lag o (all o < L_tau/2) or to lag
                        // L_tau - o (all o > L_tau/2), only the tiles around L_tau/2
                        // need the per-element choice
                        const int obase = (jb - i) * kTile;
                        const int omin = jb == i ? 1 : obase - (kTile - 1), omax = obase + kTile - 1;
                        const bool full = (jb + 1) * kTile <= Lt && (i + 1) * kTile <= Lt;
                        const int cls = (omax < half) ? 0 : (omin > half ? 1 : 2);
                        uint32_t v[64];
                        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * kTile + cbase);
#pragma unroll
                        for (int c = 0; c < 64; c += 16)
                            asm volatile(
                                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                                : "=r"(v[c + 0]), "=r"(v[c + 1]), "=r"(v[c + 2]), "=r"(v[c + 3]), "=r"(v[c + 4]),
                                  "=r"(v[c + 5]), "=r"(v[c + 6]), "=r"(v[c + 7]), "=r"(v[c + 8]), "=r"(v[c + 9]),
                                  "=r"(v[c + 10]), "=r"(v[c + 11]), "=r"(v[c + 12]), "=r"(v[c + 13]), "=r"(v[c + 14]),
                                  "=r"(v[c + 15])
                                : "r"(taddr + (uint32_t)c));
                        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                        // the accumulator is free for the tile after next
                        asm volatile("tcgen05.fence::before_thread_sync;\n");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&ctl.accempty[a]);
                        const int o0 = obase + cbase - m;  // offset of column q is o0 + q
                        if (full && cls == 0 && jb != i) {
                            // every element folds to lag o0 + q (all o < L_tau/2)
                            int *bc = binC + o0;
                            unsigned *bq = binQ + o0;
#pragma unroll
                            for (int q = 0; q < 64; ++q) {
                                const int gv = exact_f32_to_int(v[q]);
                                atomicAdd(bc + q, gv);
                                atomicAdd(bq + q, (unsigned)(gv * gv));
                            }
                        } else if (full && cls == 1) {
                            // every element folds to lag L_tau - o0 - q, the wrapped
                            // forward pair (APBC: C takes the minus sign)
                            int *bc = binC + (Lt - o0);
                            unsigned *bq = binQ + (Lt - o0);
                            if (whigh == 1) {
#pragma unroll
                                for (int q = 0; q < 64; ++q) {
                                    const int gv = exact_f32_to_int(v[q]);
                                    atomicAdd(bc - q, gv);
                                    atomicAdd(bq - q, (unsigned)(gv * gv));
                                }
                            } else {
#pragma unroll
                                for (int q = 0; q < 64; ++q) {
                                    const int gv = exact_f32_to_int(v[q]);
                                    atomicAdd(bc - q, -gv);
                                    atomicAdd(bq - q, (unsigned)(gv * gv));
                                }
                            }
                        } else if (t1 < Lt) {
#pragma unroll
                            for (int q = 0; q < 64; ++q) {
                                const int t2 = jb * kTile + cbase + q;
                                const int o = o0 + q;
                                if (t2 < Lt && o > 0) {
                                    const int gv = exact_f32_to_int(v[q]);
                                    int lag, wc, wq;
                                    if (o < half) {
                                        lag = o; wc = 1; wq = 1;
                                    } else if (o == half) {
                                        lag = half; wc = g.boundary == 1 ? 0 : 2; wq = 2;
                                    } else {
                                        lag = Lt - o; wc = whigh; wq = 1;
                                    }
                                    atomicAdd(&binC[lag], wc * gv);
                                    atomicAdd(&binQ[lag], (unsigned)(wq * gv * gv));
                                }
                            }
                        }
                    } else {
                        asm volatile("tcgen05.fence::before_thread_sync;\n");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&ctl.accempty[a]);
                    }
                }
            }
            // the unit's bins are complete: add them to the sample's int64 sums;
            // a CTA's t1 span two row blocks, so a bin holds at most 2 x 256
            // products G^2 <= 2^20 (L <= 32): 2^29, exact in 32 bits
            asm volatile("bar.sync 1, %0;\n" ::"n"(kEpilogue) : "memory");
            const int sb = sidx / 64, bit = sidx % 64;
            const int pb = sb / g.R, r = sb % g.R;
            const int pidx = p0 + pb, w = pidx / g.K, j = pidx % g.K;
            const size_t gbase = ((((size_t)r * g.W * 64) + (size_t)w * 64 + bit) * g.K + j) * nl;
            const bool write = !*(volatile int *)&ctl.abort;
            for (int l = etid; l < nl; l += kEpilogue) {
                long long c = binC[l];
                unsigned long long qv = binQ[l];
                // the diagonal (lag 0) is G(t, t) = L^2 for every t: once per sample
                if (l == 0 && h == 0) {
                    c += (long long)Lt * L2;
                    qv += (unsigned long long)Lt * L2 * L2;
                }
                if (write && c) atomicAdd(reinterpret_cast<unsigned long long *>(&g.Cacc[gbase + l]), (unsigned long long)c);
                if (write && qv) atomicAdd(reinterpret_cast<unsigned long long *>(&g.Qacc[gbase + l]), qv);
                binC[l] = 0;
                binQ[l] = 0u;
            }
            asm volatile("bar.sync 1, %0;\n" ::"n"(kEpilogue) : "memory");
        }
    } else {
        // ------------------------------------------------------------------ MMA
        const uint32_t idesc = idesc_e4m3_128x128();
        uint32_t a_par = 0u, b_par = 0u, n_t = 0;
        int bs = 0, ab = 0;
        bool issued = false;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            const int h = u % nhalf;
            for (int item = 0; item < unit_items(h, nb); ++item) {
                const int i = item_block(h, item, nb);
                const bool a_ok = mbar_wait(&ctl.afull[ab], (a_par >> ab) & 1u, &ctl.abort, wait_limit);
                const uint8_t *sAb = sA + (size_t)ab * nc * kChunkBytes;
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                for (int jb = i; jb < nb; ++jb, ++n_t) {
                    const int a = (int)(n_t & 1u);
                    bool ok = a_ok && mbar_wait(&ctl.accempty[a], ((n_t >> 1) & 1u) ^ 1u, &ctl.abort, wait_limit);
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    for (int kc = 0; kc < nc; ++kc) {
                        const uint32_t abase = smem_u32(sAb + (size_t)kc * kChunkBytes);
                        uint32_t bbase = abase;
                        if (jb != i) {
                            ok = mbar_wait(&ctl.bfull[bs], b_par, &ctl.abort, wait_limit) && ok;
                            asm volatile("tcgen05.fence::after_thread_sync;\n");
                            bbase = smem_u32(sB + (size_t)bs * kChunkBytes);
                        }
                        if (ok && lane == 0) {
#pragma unroll
                            for (int kk = 0; kk < kChunk / 32; ++kk) {
                                const uint64_t da = sdesc_sw128(abase + kk * 32);
                                const uint64_t db = sdesc_sw128(bbase + kk * 32);
                                const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                                asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                                 tmem + (uint32_t)(a * kTile)),
                                             "l"(da), "l"(db), "r"(idesc), "r"(acc));
                            }
                            issued = true;
                        }
                        if (jb != i) {
                            if (lane == 0) mma_commit(&ctl.bempty[bs]);
                            if (++bs == nstages) {
                                bs = 0;
                                b_par ^= 1u;
                            }
                        }
                        __syncwarp();
                    }
                    if (lane == 0) mma_commit(&ctl.accfull[a]);
                    __syncwarp();
                }
                if (lane == 0) mma_commit(&ctl.aempty[ab]);
                __syncwarp();
                a_par ^= 1u << ab;
                if (++ab == nabuf) ab = 0;
            }
        }
        // every MMA issued has completed before the tensor memory is released
        // (a commit tracks all earlier MMAs of the issuing thread)
        if (lane == 0) {
            mma_commit(&ctl.done);
            if (issued) {
                uint32_t done = 0;
                for (unsigned it = 0; it < kSpinLimit && !done; ++it)
                    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
                                 : "=r"(done)
                                 : "r"(smem_u32(&ctl.done))
                                 : "memory");
                if (!done) ctl.abort = 1;
            }
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
    if (tid == 0 && ctl.abort) atomicExch(status, DEVERR_TIMEOUT);
}

namespace {

size_t gram_tc_smem_bytes(const Group &g, int nstages, int nabuf) {
    const int nc = (g.L * g.L + kChunk - 1) / kChunk;
    return 1024 + (size_t)(nabuf * nc + nstages) * kChunkBytes + 2 * sizeof(int) * (size_t)g.nlag;
}

constexpr size_t kSmemLimit = 227 * 1024 - 256;  // dynamic + the static control block

// Shared-memory plan: two A buffers (the next row block is expanded while the
// last tiles of the current one are multiplied) with at least four B stages
// where that fits, else one A buffer; as many B stages as fit, up to six.
struct TcPlan {
    int nstages, nabuf;
};

TcPlan gram_tc_plan(const Group &g) {
    for (int nabuf = 2; nabuf >= 1; --nabuf)
        for (int s = kMaxStages; s >= (nabuf == 2 ? 4 : 2); --s)
            if (gram_tc_smem_bytes(g, s, nabuf) <= kSmemLimit) return {s, nabuf};
    return {0, 0};
}

}  // namespace

bool gram_tc_fits(const Group &g) { return gram_tc_plan(g).nstages >= 2; }

cudaError_t launch_gram_tc(const Group &g, int p0, int npairs, const uint64_t *P, int *status, unsigned wait_limit,
                           cudaStream_t st) {
    const TcPlan plan = gram_tc_plan(g);
    if (plan.nstages < 2) return cudaErrorInvalidValue;
    const size_t sm = gram_tc_smem_bytes(g, plan.nstages, plan.nabuf);
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nsamples = npairs * g.R * 64;
    const int nb = (g.Ltau + kTile - 1) / kTile;
    const long long nunits = (long long)nsamples * ((nb + 1) / 2);
    const int grid = (int)(nunits < nsm ? nunits : nsm);
    count_launches(1);
    k_gram_tc<<<grid, kThreads, sm, st>>>(g, p0, P, nsamples, plan.nstages, plan.nabuf, status, wait_limit);
    return cudaGetLastError();
}

}  // namespace qsg
