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
//   producers (8 warps) load the x-packed bit rows of the transposed scratch
//     one block ahead into registers and expand them to E4M3 +-1 (0 for
//     padding) in shared memory, K-major with the 128-byte swizzle, sites in a
//     bit-interleaved order shared by A and B: the row block A of an item in
//     128-site chunks, each with its own full/empty barrier pair (so the next
//     item's A is written chunk by chunk as the last tile of the current one
//     releases it), and B two column blocks at a time in 32 KB stages (256
//     rows x 128 sites);
//   one thread issues the MMAs: the diagonal tile (i, i) with N = 128 and
//     B = A, then the column-block pairs (i, j), (i, j + 1) as one N = 256
//     MMA per 32-site step (a single block when the count is odd), into two
//     256-column tensor-memory accumulators, so the next tile is multiplied
//     while the last one is folded.  Issue is nearly synchronous with the
//     tensor pipe, so the issuing thread does nothing between MMAs but wait
//     for a stage every four of them;
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
constexpr int kStageBytes = 2 * kChunkBytes; // 32 KB per B stage (two column blocks)
constexpr int kMaxStages = 6;                // B stages at most
constexpr int kProducers = 256;              // warps 0-7: one thread per B stage row
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

// Instruction descriptor: D = FP32, A = B = E4M3, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_e4m3(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

struct Ctl {
    uint64_t bfull[kMaxStages], bempty[kMaxStages];  // B stage written / multiplied
    uint64_t afull[kMaxNc], aempty[kMaxNc];          // A chunk written / multiplied
    uint64_t accfull[2], accempty[2];                // accumulator computed / folded
    uint64_t done;                                   // every MMA of the CTA completed
    uint32_t tmem;
    int abort;  // a wait gave up: every role skips its work and runs out its loops
};

// Wait for the phase of the given parity; false (and the abort flag set) when
// `limit` polls are used up, or when another thread has given up already (the
// flag is read every 64 polls, after the barrier itself).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *abort, unsigned limit) {
    const uint32_t a = smem_u32(bar);
    volatile int *ab = abort;
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 63u) == 63u && *ab) return false;
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

// FP32 accumulator holding an integer |x| < 2^22 -> int32 with one add: in
// [2^23, 2^24) the FP32 spacing is 1, so x + 1.5 * 2^23 is exact and its bit
// pattern is that of 1.5 * 2^23 plus x.
__device__ __forceinline__ int exact_f32_to_int(uint32_t bits) {
    return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}


__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// The work of one CTA: units u = blockIdx.x + n gridDim.x; unit u is sample
// u / nhalf, row blocks h = u % nhalf and nb - 1 - h (one block when equal).
// Within a unit the blocks are items; item i has the diagonal tile (i, i) and
// the column-block pairs (i, jp), (i, jp + 1), jp = i + 1, i + 3, ...
__device__ __forceinline__ int item_block(int h, int item, int nb) { return item ? nb - 1 - h : h; }
__device__ __forceinline__ int unit_items(int h, int nb) { return nb - 1 - h != h ? 2 : 1; }

// The producers' block sequence: per item the A block i, then the pairs.
struct Seq {
    int u, sidx, h, item, i, jp;
    bool isA, valid;
};

__device__ __forceinline__ void seq_unit(Seq &c, int nunits, int nhalf) {
    c.valid = c.u < nunits;
    c.sidx = c.u / nhalf;
    c.h = c.u - c.sidx * nhalf;
    c.item = 0;
    c.i = c.h;
    c.isA = true;
    c.jp = c.h;
}

__device__ __forceinline__ void seq_next(Seq &c, int nunits, int nhalf, int nb) {
    if (c.isA) {
        c.isA = false;
        c.jp = c.i + 1;
        if (c.jp < nb) return;
    } else {
        c.jp += 2;
        if (c.jp < nb) return;
    }
    if (++c.item >= unit_items(c.h, nb)) {
        c.u += gridDim.x;
        seq_unit(c, nunits, nhalf);
        return;
    }
    c.i = item_block(c.h, c.item, nb);
    c.isA = true;
    c.jp = c.i;
}

// Bit words of producer thread pt for block c, 0 outside the lattice and past
// L_tau.  A block: w[kc] = word 2 kc + (pt >> 7) of row (pt & 127) of block
// i.  Pair: w[2 kc + hh] = word 2 kc + hh of stage row pt (rows 0..127 are
// block jp, rows 128..255 block jp + 1).
template <int NC>
__device__ __forceinline__ void load_seq(const Seq &c, const uint64_t *__restrict__ P, int Lt, int nwx, int pt,
                                         uint64_t (&w)[2 * NC]) {
    const size_t sbase = (size_t)(c.valid ? c.sidx : 0) * Lt;
    if (c.isA) {
        const int row = pt & 127, hh = pt >> 7;
        const int t = c.i * kTile + row;
        const bool in = c.valid && t < Lt;
        const uint64_t *src = P + (sbase + (in ? t : 0)) * nwx + hh;
#pragma unroll
        for (int kc = 0; kc < NC; ++kc) w[kc] = (in && 2 * kc + hh < nwx) ? __ldg(src + 2 * kc) : 0ull;
    } else {
        const int t = (c.jp + (pt >> 7)) * kTile + (pt & 127);
        const bool in = c.valid && t < Lt;
        const uint64_t *src = P + (sbase + (in ? t : 0)) * nwx;
#pragma unroll
        for (int kc = 0; kc < NC; ++kc)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
                w[2 * kc + hh] = (in && 2 * kc + hh < nwx) ? __ldg(src + 2 * kc + hh) : 0ull;
    }
}

// Fold the 64 columns cbase .. cbase + 63 of row m of tile (i, jb) into the
// lag bins.  Most tiles map every element to lag o (all o < L_tau/2) or to
// lag L_tau - o (all o > L_tau/2); only the tiles around L_tau/2 and those
// past L_tau need the per-element choice.
__device__ __forceinline__ void fold_slice(const uint32_t (&v)[64], int i, int jb, int m, int cbase, int Lt, int half,
                                           int boundary, int *binC, unsigned *binQ) {
    const int whigh = boundary == 1 ? -1 : 1;
    const int t1 = i * kTile + m;
    const int obase = (jb - i) * kTile;
    const int omin = jb == i ? 1 : obase - (kTile - 1), omax = obase + kTile - 1;
    const bool full = (jb + 1) * kTile <= Lt && (i + 1) * kTile <= Lt;
    const int cls = (omax < half) ? 0 : (omin > half ? 1 : 2);
    const int o0 = obase + cbase - m;  // offset of column q is o0 + q
    if (full && cls == 0 && jb != i) {
        int *bc = binC + o0;
        unsigned *bq = binQ + o0;
#pragma unroll
        for (int q = 0; q < 64; ++q) {
            const int gv = exact_f32_to_int(v[q]);
            atomicAdd(bc + q, gv);
            atomicAdd(bq + q, (unsigned)(gv * gv));
        }
    } else if (full && cls == 1) {
        // the wrapped forward pair: lag L_tau - o0 - q (APBC: C takes the minus sign)
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
                    lag = half; wc = boundary == 1 ? 0 : 2; wq = 2;
                } else {
                    lag = Lt - o; wc = whigh; wq = 1;
                }
                atomicAdd(&binC[lag], wc * gv);
                atomicAdd(&binQ[lag], (unsigned)(wq * gv * gv));
            }
        }
    }
}

// 64 consecutive accumulator columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
#pragma unroll
    for (int c = 0; c < 64; c += 16)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[c + 0]), "=r"(v[c + 1]), "=r"(v[c + 2]), "=r"(v[c + 3]), "=r"(v[c + 4]), "=r"(v[c + 5]),
              "=r"(v[c + 6]), "=r"(v[c + 7]), "=r"(v[c + 8]), "=r"(v[c + 9]), "=r"(v[c + 10]), "=r"(v[c + 11]),
              "=r"(v[c + 12]), "=r"(v[c + 13]), "=r"(v[c + 14]), "=r"(v[c + 15])
            : "r"(taddr + (uint32_t)c));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

}  // namespace

// P: [sample][Ltau][nwx] transposed bits of the batch (sample = (pair, r, bit)).
// NC = 128-site chunks of a row (L^2 / 128 rounded up).
template <int NC>
__global__ void __launch_bounds__(kThreads, 1)
    k_gram_tc(Group g, int p0, const uint64_t *__restrict__ P, int nsamples, int nstages, int *status,
              unsigned wait_limit) {
    extern __shared__ __align__(16) uint8_t dyn_raw[];
    uint8_t *dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);
    __shared__ Ctl ctl;
    const int Lt = g.Ltau, L2 = g.L * g.L, half = Lt / 2, nl = g.nlag, nwx = g.nwx;
    const int nb = (Lt + kTile - 1) / kTile, nhalf = (nb + 1) / 2;
    const int nunits = nsamples * nhalf;
    uint8_t *sA = dyn;                            // NC chunks of 128 rows x 128 sites
    uint8_t *sB = sA + (size_t)NC * kChunkBytes;  // stages of 256 rows x 128 sites
    int *binC = reinterpret_cast<int *>(sB + (size_t)nstages * kStageBytes);
    unsigned *binQ = reinterpret_cast<unsigned *>(binC + nl);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&ctl.bfull[s])), "r"(kProducerWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&ctl.bempty[s])));
        }
        for (int k = 0; k < kMaxNc; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&ctl.afull[k])), "r"(kProducerWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&ctl.aempty[k])));
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
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(&ctl.tmem)));
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

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers
        // the bit words of the next block are loaded into registers while the
        // current one is expanded; one chunk loop serves both kinds of block:
        // an A block's thread writes word tid >> 7 of row tid & 127, a pair
        // block's thread both words of stage row tid (none past a single
        // last block)
        Seq cur, nxt;
        cur.u = blockIdx.x;
        seq_unit(cur, nunits, nhalf);
        uint64_t wc[2 * NC], wn[2 * NC];
        load_seq<NC>(cur, P, Lt, nwx, tid, wc);
        // the first use of a buffer waits for the phase before the first
        // (complete at initialisation)
        uint32_t a_ph = 1u, b_par = 1u;
        int s = 0;
        while (cur.valid) {
            nxt = cur;
            seq_next(nxt, nunits, nhalf, nb);
            load_seq<NC>(nxt, P, Lt, nwx, tid, wn);
            const bool isA = cur.isA;
            const bool pair = cur.jp + 1 < nb;
            const int row = isA ? (tid & 127) : tid, hh0 = isA ? (tid >> 7) : 0;
            const int nw = isA ? 1 : ((pair || tid < kTile) ? 2 : 0);
            const int t = isA ? cur.i * kTile + row : (cur.jp + (tid >> 7)) * kTile + (tid & 127);
            // the chunk loop stays rolled (the three roles' code shares the
            // instruction cache): the words of chunk kc are always in wc[0],
            // wc[1] (an A block's in wc[0]), and the array shifts after a chunk
#pragma unroll 1
            for (int kc = 0; kc < NC; ++kc) {
                const bool ok = isA ? mbar_wait(&ctl.aempty[kc], a_ph, &ctl.abort, wait_limit)
                                    : mbar_wait(&ctl.bempty[s], b_par, &ctl.abort, wait_limit);
                uint8_t *rowp = isA ? sA + (size_t)kc * kChunkBytes + row * kChunk
                                    : sB + (size_t)s * kStageBytes + row * kChunk;
                const uint64_t w0 = wc[0], w1 = wc[1];
                if (ok) {
#pragma unroll 1
                    for (int k = 0; k < nw; ++k) {
                        const int hh = hh0 + k;
                        // a word past the lattice's last site is never read (the
                        // MMAs of the last chunk stop at its last word with a site)
                        if (L2 - kc * kChunk - 64 * hh > 0)
                            expand_word(rowp, k ? w1 : w0, t < Lt ? L2 - kc * kChunk - 64 * hh : 0, hh, row);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();  // the warp's rows are written: one arrival per warp
                if (lane == 0) mbar_arrive(isA ? &ctl.afull[kc] : &ctl.bfull[s]);
                if (!isA && ++s == nstages) {
                    s = 0;
                    b_par ^= 1u;
                }
                const int sh = isA ? 1 : 2;  // words per chunk of this kind of block
#pragma unroll
                for (int k = 0; k < 2 * NC - 2; ++k) wc[k] = sh == 1 ? wc[k + 1] : wc[k + 2];
            }
            if (isA) a_ph ^= 1u;
#pragma unroll
            for (int k = 0; k < 2 * NC; ++k) wc[k] = wn[k];
            cur = nxt;
        }
    } else if (warp < kMmaWarp) {
        // ------------------------------------------------------------- epilogue
        const int etid = tid - kProducers;
        const int quad = warp & 3;                                  // TMEM lanes 32 quad .. 32 quad + 31
        const int cbase = ((warp - kProducerWarps) >> 2) * 64;     // column half of a 128-column tile
        const int m = quad * 32 + lane;                             // tile row
        uint32_t n_t = 0;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
            const int sidx = u / nhalf, h = u % nhalf;
            for (int item = 0; item < unit_items(h, nb); ++item) {
                const int i = item_block(h, item, nb);
                // the MMA's tile order: (i, i), then the pairs from jp = i + 1
                for (int jp = i; jp < nb; jp = (jp == i ? i + 1 : jp + 2), ++n_t) {
                    const int nsub = (jp != i && jp + 1 < nb) ? 2 : 1;
                    const int a = (int)(n_t & 1u);
                    // warp-uniform: the tensor-memory loads below are .sync.aligned
                    const bool ok =
                        __all_sync(0xFFFFFFFFu, mbar_wait(&ctl.accfull[a], (n_t >> 1) & 1u, &ctl.abort, wait_limit));
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    if (ok) {
                        for (int sub = 0; sub < nsub; ++sub) {
                            uint32_t v[64];
                            tmem_ld64(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * 256 + sub * kTile + cbase),
                                      v);
                            if (sub == nsub - 1) {
                                // the accumulator is free for the tile after next
                                asm volatile("tcgen05.fence::before_thread_sync;\n");
                                __syncwarp();
                                if (lane == 0) mbar_arrive(&ctl.accempty[a]);
                            }
                            fold_slice(v, i, jp + sub, m, cbase, Lt, half, g.boundary, binC, binQ);
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
        // one thread issues every MMA; after the last tile of an item uses an
        // A chunk, a commit frees that chunk for the next item's A block
        if (lane == 0) {
            const uint32_t id128 = idesc_e4m3(128), id256 = idesc_e4m3(256);
            // 32-site steps of the last chunk: those of its 64-site words that
            // hold a lattice site (the bit-interleaved order spreads a word's
            // sites over its whole 64-byte span)
            const int nk_last = min(kChunk / 32, 2 * ((L2 - (NC - 1) * kChunk + 63) / 64));
            const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
            uint32_t a_par = 0u, b_par = 0u, n_t = 0;
            int bs = 0;
            bool issued = false;
            for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
                const int h = u % nhalf;
                for (int item = 0; item < unit_items(h, nb); ++item) {
                    const int i = item_block(h, item, nb);
                    {  // the diagonal tile: B = A, 128 columns
                        const bool last = i + 1 >= nb;
                        const int a = (int)(n_t & 1u);
                        bool ok = mbar_wait(&ctl.accempty[a], ((n_t >> 1) & 1u) ^ 1u, &ctl.abort, wait_limit);
                        asm volatile("tcgen05.fence::after_thread_sync;\n");
                        const uint32_t d = tmem + (uint32_t)(a * 256);
#pragma unroll 1  // rolled: the three roles' code shares the instruction cache
                        for (int kc = 0; kc < NC; ++kc) {
                            ok = mbar_wait(&ctl.afull[kc], a_par, &ctl.abort, wait_limit) && ok;
                            asm volatile("tcgen05.fence::after_thread_sync;\n");
                            if (ok) {
                                const uint32_t ab = sA0 + kc * kChunkBytes;
                                const int nk = kc == NC - 1 ? nk_last : kChunk / 32;
#pragma unroll
                                for (int kk = 0; kk < kChunk / 32; ++kk)
                                    if (kk < nk)
                                        mma_f8(d, sdesc_sw128(ab + kk * 32), sdesc_sw128(ab + kk * 32), id128,
                                               (kc > 0 || kk > 0) ? 1u : 0u);
                                issued = true;
                            }
                            if (last) mma_commit(&ctl.aempty[kc]);
                        }
                        mma_commit(&ctl.accfull[a]);
                        ++n_t;
                    }
                    for (int jp = i + 1; jp < nb; jp += 2) {  // column blocks jp and jp + 1
                        const bool pair = jp + 1 < nb, last = jp + 2 >= nb;
                        const int a = (int)(n_t & 1u);
                        bool ok = mbar_wait(&ctl.accempty[a], ((n_t >> 1) & 1u) ^ 1u, &ctl.abort, wait_limit);
                        asm volatile("tcgen05.fence::after_thread_sync;\n");
                        const uint32_t d = tmem + (uint32_t)(a * 256);
                        const uint32_t idesc = pair ? id256 : id128;
#pragma unroll 1  // rolled: the three roles' code shares the instruction cache
                        for (int kc = 0; kc < NC; ++kc) {
                            ok = mbar_wait(&ctl.bfull[bs], b_par, &ctl.abort, wait_limit) && ok;
                            asm volatile("tcgen05.fence::after_thread_sync;\n");
                            if (ok) {
                                const uint32_t ab = sA0 + kc * kChunkBytes, bb = sB0 + bs * kStageBytes;
                                const int nk = kc == NC - 1 ? nk_last : kChunk / 32;
#pragma unroll
                                for (int kk = 0; kk < kChunk / 32; ++kk)
                                    if (kk < nk)
                                        mma_f8(d, sdesc_sw128(ab + kk * 32), sdesc_sw128(bb + kk * 32), idesc,
                                               (kc > 0 || kk > 0) ? 1u : 0u);
                                issued = true;
                            }
                            mma_commit(&ctl.bempty[bs]);
                            if (last) mma_commit(&ctl.aempty[kc]);
                            if (++bs == nstages) {
                                bs = 0;
                                b_par ^= 1u;
                            }
                        }
                        mma_commit(&ctl.accfull[a]);
                        ++n_t;
                    }
                    a_par ^= 1u;
                }
            }
            // every MMA issued has completed before the tensor memory is released
            // (a commit tracks all earlier MMAs of the issuing thread)
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
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
    if (tid == 0 && ctl.abort) atomicExch(status, DEVERR_TIMEOUT);
}

namespace {

constexpr size_t kSmemLimit = 227 * 1024 - 256;  // dynamic + the static control block

size_t gram_tc_smem_bytes(const Group &g, int nc, int nstages) {
    return 1024 + (size_t)nc * kChunkBytes + (size_t)nstages * kStageBytes + 2 * sizeof(int) * (size_t)g.nlag;
}

// As many B stages as fit, up to six; at least two.
int gram_tc_stages(const Group &g) {
    const int nc = (g.L * g.L + kChunk - 1) / kChunk;
    if (nc < 1 || nc > kMaxNc) return 0;
    for (int s = kMaxStages; s >= 2; --s)
        if (gram_tc_smem_bytes(g, nc, s) <= kSmemLimit) return s;
    return 0;
}

template <int NC>
cudaError_t launch_nc(const Group &g, int p0, int nsamples, int nstages, const uint64_t *P, int *status,
                      unsigned wait_limit, int nsm, cudaStream_t st) {
    const size_t sm = gram_tc_smem_bytes(g, NC, nstages);
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nb = (g.Ltau + kTile - 1) / kTile;
    const long long nunits = (long long)nsamples * ((nb + 1) / 2);
    const int grid = (int)(nunits < nsm ? nunits : nsm);
    count_launches(1);
    k_gram_tc<NC><<<grid, kThreads, sm, st>>>(g, p0, P, nsamples, nstages, status, wait_limit);
    return cudaGetLastError();
}

}  // namespace

bool gram_tc_fits(const Group &g) { return gram_tc_stages(g) >= 2; }

cudaError_t launch_gram_tc(const Group &g, int p0, int npairs, const uint64_t *P, int *status, unsigned wait_limit,
                           cudaStream_t st) {
    const int nstages = gram_tc_stages(g);
    if (nstages < 2) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nsamples = npairs * g.R * 64;
    switch ((g.L * g.L + kChunk - 1) / kChunk) {
        case 1: return launch_nc<1>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        case 2: return launch_nc<2>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        case 3: return launch_nc<3>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        case 4: return launch_nc<4>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        case 5: return launch_nc<5>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        case 6: return launch_nc<6>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        case 7: return launch_nc<7>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
        default: return launch_nc<8>(g, p0, nsamples, nstages, P, status, wait_limit, nsm, st);
    }
}

}  // namespace qsg
