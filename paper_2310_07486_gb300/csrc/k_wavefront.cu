// k_wavefront.cu -- one full checkerboard sweep (colour 0 then colour 1) in a
// single pass over HBM: every spin word is read once and written once.
//
// A work unit is one slot and one chunk of C consecutive tau planes [a, b).
// The unit streams its planes through a ring of 16 shared-memory planes filled
// by cp.async about eight planes ahead.  It updates the colour-0 sites of
// plane tau while their colour-1 neighbours in planes tau-1, tau, tau+1 are
// still the old ones, and the colour-1 sites of plane tau-1 once their
// colour-0 neighbours in planes tau-2, tau-1, tau are new: the order of a
// colour-0 half sweep followed by a colour-1 half sweep.
//
// The colour-1 sites of the first plane of a chunk need the new colour 0 of the
// previous chunk's last plane, and vice versa, so the colour-1 sites of planes
// a-1 and a are deferred: whichever of the two units adjacent to the boundary
// finishes second updates them (an atomic arrival counter, no waiting).
//
// Thread layout: a thread owns two neighbouring columns (x0, x0+1) of row y,
// with pairs starting at x = y & 1, so that on every plane the colour-0 column
// is the same (x0 on even planes, x0+1 on odd ones) for every thread (no
// divergence), and one Philox call per 2 x 2 (x, tau) block serves the four
// updates of that block.
//
// Shared-memory planes are stored split by checkerboard class: sites with
// (x + y) even first, then (x + y) odd, each as [y][x/2].  Column x0 of every
// thread is class "even" at index c = thread index, so the active sites of a
// step and their neighbours are read by consecutive threads from consecutive
// words.
#include <type_traits>

#include "qsg_launch.h"
#include "qsg_sweep.cuh"

namespace qsg {

namespace {

using namespace sweep;

// Per-thread offsets in the class-split shared-memory plane.
struct Thr {
    int o0, o1;        // own columns x0 (even class, = thread index) and x0+1 (odd class)
    int l0, u0, d0;    // neighbours of x0: left, up, down (odd class)
    int r1, u1, d1;    // neighbours of x0+1: right, up, down (even class)
    int dA, dB;        // where global words 2c and 2c+1 of a plane land
    int x0, y;         // coordinates of column x0
    uint32_t qrow;     // Philox block index within a tau pair
};

__device__ __forceinline__ Thr make_thr(int L, int c) {
    const int half = L / 2, H = L * L / 2;
    const int y = c / half, xh = c % half;
    const int x0 = 2 * xh + (y & 1);
    const int x1 = x0 + 1 == L ? 0 : x0 + 1;
    const int x0m = x0 == 0 ? L - 1 : x0 - 1;
    const int x1p = x1 + 1 == L ? 0 : x1 + 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    Thr t;
    t.o0 = c;
    t.o1 = H + y * half + (x1 >> 1);
    t.l0 = H + y * half + (x0m >> 1);
    t.u0 = H + yp * half + xh;
    t.d0 = H + ym * half + xh;
    t.r1 = y * half + (x1p >> 1);
    t.u1 = yp * half + (x1 >> 1);
    t.d1 = ym * half + (x1 >> 1);
    t.dA = (y & 1) * H + c;        // global word 2c = site (2 (c % half), y)
    t.dB = (1 - (y & 1)) * H + c;  // global word 2c+1
    t.x0 = x0;
    t.y = y;
    t.qrow = (uint32_t)c;
    return t;
}

// Colour-1 sites of the two planes around chunk boundary pb: (x0, pb-1) and
// (x0+1, pb); all their neighbours are final colour-0 sites.  Spins are read
// from global memory (bypassing L1, the neighbouring unit wrote them); the
// couplings come from the class-split shared copy.
template <int ALGO>
__device__ __forceinline__ void boundary_update(const Group &g, const Thr &t, uint64_t *Sg, const uint64_t *sJx,
                                                const uint64_t *sJy, int pb, const Thresh &T, uint32_t sweep,
                                                uint32_t slot, uint32_t k0, uint32_t k1) {
    const int L = g.L, L2 = L * L, Lt = g.Ltau, half = L / 2;
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;
    const int x0 = t.x0, y = t.y;
    const int x1 = x0 + 1 == L ? 0 : x0 + 1;
    const int x0m = x0 == 0 ? L - 1 : x0 - 1, x1p = x1 + 1 == L ? 0 : x1 + 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int n0 = y * L + x0, n1 = y * L + x1;
    {
        const int p = pb == 0 ? Lt - 1 : pb - 1;  // odd plane: x0 is colour 1
        const uint64_t *P = Sg + (size_t)p * L2;
        const uint64_t *Pp = Sg + (size_t)(p + 1 == Lt ? 0 : p + 1) * L2;
        const uint64_t *Pm = Sg + (size_t)(p - 1) * L2;
        const uint64_t fp = p == Lt - 1 ? apbc : 0ull;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(L * half) + t.qrow, sweep, slot, tag),
                                      k0, k1);
        const uint64_t v = update_site<ALGO>(__ldcg(P + n0), __ldcg(P + n1), __ldcg(P + y * L + x0m),
                                             __ldcg(P + yp * L + x0), __ldcg(P + ym * L + x0), __ldcg(Pp + n0) ^ fp,
                                             __ldcg(Pm + n0), sJx[t.o0], sJx[t.l0], sJy[t.o0], sJy[t.d0], r.z, T);
        Sg[(size_t)p * L2 + n0] = v;
    }
    {
        const int p = pb;  // even plane: x0+1 is colour 1
        const uint64_t *P = Sg + (size_t)p * L2;
        const uint64_t *Pp = Sg + (size_t)(p + 1) * L2;
        const uint64_t *Pm = Sg + (size_t)(p == 0 ? Lt - 1 : p - 1) * L2;
        const uint64_t fm = p == 0 ? apbc : 0ull;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(L * half) + t.qrow, sweep, slot, tag),
                                      k0, k1);
        const uint64_t v = update_site<ALGO>(__ldcg(P + n1), __ldcg(P + y * L + x1p), __ldcg(P + n0),
                                             __ldcg(P + yp * L + x1), __ldcg(P + ym * L + x1), __ldcg(Pp + n1),
                                             __ldcg(Pm + n1) ^ fm, sJx[t.o1], sJx[t.o0], sJy[t.o1], sJy[t.d1], r.y, T);
        Sg[(size_t)p * L2 + n1] = v;
    }
}

}  // namespace

// SLOT: shared-memory words per ring plane (>= L^2), a compile-time stride so
// that every ring address is a register plus an immediate.
//
// Schedule.  The only dependence between threads is that all colour-0
// updates of a plane precede any colour-1 update of it (the colour-1 sites
// read their colour-0 neighbours, the colour-0 sites must read the old
// colour 1).  Updates of one thread along its own columns are ordered by the
// program.  A super step (q = a + 2m) therefore runs
//     colour 0 of planes q, q+1  |barrier|  colour 1 of planes q-1, q
// with one barrier per two planes.
// One work unit (slot s, chunk ch of C planes) run by the threads that share
// `ring` (kRing * SLOT + 2 L^2 words of shared memory); threads with
// active == false only take part in the barriers.  do_boundary is one int of
// shared memory for this unit; the arrival counter of the boundary at the
// start of chunk ch is arrivals[s * astride + ch].
template <int ALGO, int SLOT, bool JREG = false>
__device__ __forceinline__ void wavefront_unit(const Group &g, const int C, const int astride, const int s,
                                               const int ch,
                                               const bool active, const int c, uint64_t *ring, int *do_boundary,
                                               const uint32_t sweep, const uint32_t k0, const uint32_t k1,
                                               unsigned *__restrict__ arrivals) {
    const int L = g.L, L2 = L * L, Lt = g.Ltau, half = L / 2;
    const int a = ch * C, b = a + C;
    const int w = s / (g.R * g.K), j = s % g.K;
    uint64_t *sJx = ring + kRing * SLOT, *sJy = sJx + L2;
    uint64_t *Sg = g.S + (size_t)s * g.N;
    const Thr t = make_thr(L, c);
    if (active) {
        // couplings of word-group w, stored class-split like the spin planes
        const uint64_t *gJx = g.Jx + (size_t)w * L2, *gJy = g.Jy + (size_t)w * L2;
        sJx[t.dA] = gJx[2 * c];
        sJx[t.dB] = gJx[2 * c + 1];
        sJy[t.dA] = gJy[2 * c];
        sJy[t.dB] = gJy[2 * c + 1];
    }
    Thresh T;
#pragma unroll
    for (int n = 0; n < 7; ++n) T.t[n] = g.thr[j * 16 + (ALGO == 0 ? n % 3 : 8 + n)];
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint32_t qstride = (uint32_t)(L * half);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;

    // plane p of the chunk lives in ring slot (p - a + 1) & 15.  `edge` is false
    // in the interior of the chunk, where every plane issued lies in [a, b)
    // and needs no wrap.
    auto issue_plane = [&](int p, uint64_t *dst, auto edge) {
        constexpr bool E = decltype(edge)::value;
        if (active && (!E || p <= b)) {
            const int gp = !E ? p : (p < 0 ? p + Lt : (p >= Lt ? p - Lt : p));
            const uint64_t *src = Sg + (size_t)gp * L2 + 2 * c;
            cp_async8(dst + t.dA, src);
            cp_async8(dst + t.dB, src + 1);
        }
    };
    auto writeback = [&](int p, const uint64_t *src) {
        *reinterpret_cast<ulonglong2 *>(Sg + (size_t)p * L2 + 2 * c) = make_ulonglong2(src[t.dA], src[t.dB]);
    };

    // prologue: planes a-1 .. a+7 in slots 0 .. 8
#pragma unroll
    for (int i = 0; i < 9; ++i) issue_plane(a - 1 + i, ring + i * SLOT, std::true_type{});
    cp_commit();
    uint4 rcur = philox4x32_10(make_uint4((uint32_t)(a >> 1) * qstride + t.qrow, sweep, (uint32_t)s, tag), k0, k1);
    uint32_t carry = 0;
    cp_wait<0>();
    __syncthreads();
    // own columns at planes q-2 .. q+2 of super step m, register index (p - a) & 7
    uint64_t W0[8], W1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) W0[i] = W1[i] = 0;
    W0[7] = ring[0 * SLOT + t.o0];  // plane a-1
    W1[7] = ring[0 * SLOT + t.o1];
    W0[0] = ring[1 * SLOT + t.o0];  // plane a
    // couplings of the thread's two sites (JREG: held in registers for the
    // whole chunk instead of re-read from shared memory every super step)
    uint64_t Jr0 = 0, Jl0 = 0, Ju0 = 0, Jd0 = 0, Jr1 = 0, Ju1 = 0, Jd1 = 0;
    if (JREG) {
        Jr0 = sJx[t.o0];
        Jl0 = sJx[t.l0];
        Ju0 = sJy[t.o0];
        Jd0 = sJy[t.d0];
        Jr1 = sJx[t.o1];
        Ju1 = sJy[t.o1];
        Jd1 = sJy[t.d1];
    }
    W1[0] = ring[1 * SLOT + t.o1];

// ring slot of plane a + p_rel; inside the loop p_rel is taken modulo 16
// (base - a is a multiple of 16), which makes the slot a compile-time constant
#define QSG_SLOT(p_rel) (ring + (((p_rel) + 1) & (kRing - 1)) * SLOT)
#define QSG_SUPER(MM)                                                                                             \
    {                                                                                                             \
        constexpr int Q = 2 * (MM);            /* q - base, 0..14 */                                             \
        constexpr int R0 = Q & 7, RP1 = (Q + 1) & 7, RP2 = (Q + 2) & 7, RM1 = (Q + 7) & 7, RM2 = (Q + 6) & 7;    \
        const int q = base + Q;                                                                                   \
        /* own columns of planes q+1, q+2 (landed and made visible before the last barrier) */                   \
        W0[RP1] = QSG_SLOT(Q + 1)[t.o0];                                                                          \
        W1[RP1] = QSG_SLOT(Q + 1)[t.o1];                                                                          \
        W0[RP2] = QSG_SLOT(Q + 2)[t.o0];                                                                          \
        W1[RP2] = QSG_SLOT(Q + 2)[t.o1];                                                                          \
        /* prefetch planes q+8, q+9 */                                                                            \
        issue_plane(q + 8, QSG_SLOT(Q + 8), std::integral_constant<bool, EDGE>{});                                \
        issue_plane(q + 9, QSG_SLOT(Q + 9), std::integral_constant<bool, EDGE>{});                                \
        cp_commit();                                                                                              \
        const uint64_t jr0 = JREG ? Jr0 : sJx[t.o0], jl0 = JREG ? Jl0 : sJx[t.l0];                                 \
        const uint64_t ju0 = JREG ? Ju0 : sJy[t.o0], jd0 = JREG ? Jd0 : sJy[t.d0];                                 \
        const uint64_t jr1 = JREG ? Jr1 : sJx[t.o1], ju1 = JREG ? Ju1 : sJy[t.o1], jd1 = JREG ? Jd1 : sJy[t.d1];   \
        const uint4 r = rcur;                                                                                     \
        if (active) {                                                                                             \
            /* colour 0 of plane q (column x0) and of plane q+1 (column x0+1) */                                  \
            uint64_t *pq = QSG_SLOT(Q);                                                                           \
            uint64_t *pq1 = QSG_SLOT(Q + 1);                                                                      \
            W0[R0] = update_site<ALGO>(W0[R0], W1[R0], pq[t.l0], pq[t.u0], pq[t.d0], W0[RP1],                     \
                                       W0[RM1] ^ (EDGE && q == 0 ? apbc : 0ull), jr0, jl0, ju0, jd0, r.x, T);     \
            pq[t.o0] = W0[R0];                                                                                    \
            W1[RP1] = update_site<ALGO>(W1[RP1], pq1[t.r1], W0[RP1], pq1[t.u1], pq1[t.d1],                        \
                                        W1[RP2] ^ (EDGE && q + 1 == Lt - 1 ? apbc : 0ull), W1[R0], jr1, jr0, ju1, \
                                        jd1,                                                                      \
                                        r.w, T);                                                                  \
            pq1[t.o1] = W1[RP1];                                                                                  \
        }                                                                                                         \
        /* planes <= q+5 must have landed before the barrier (the next super step reads up to q+4) */            \
        cp_wait<2>();                                                                                             \
        __syncthreads();                                                                                          \
        rcur = philox4x32_10(make_uint4((uint32_t)((q + 2) >> 1) * qstride + t.qrow, sweep, (uint32_t)s, tag),    \
                             k0, k1);                                                                             \
        if (active) {                                                                                             \
            if (!EDGE || q >= a + 2) {                                                                            \
                /* colour 1 of plane q-1 (column x0) and of plane q (column x0+1) */                              \
                uint64_t *pm = QSG_SLOT(Q - 1);                                                                   \
                uint64_t *pq = QSG_SLOT(Q);                                                                       \
                W0[RM1] = update_site<ALGO>(W0[RM1], W1[RM1], pm[t.l0], pm[t.u0], pm[t.d0], W0[R0], W0[RM2],      \
                                            jr0, jl0, ju0, jd0, carry, T);                                        \
                pm[t.o0] = W0[RM1];                                                                               \
                W1[R0] = update_site<ALGO>(W1[R0], pq[t.r1], W0[R0], pq[t.u1], pq[t.d1], W1[RP1], W1[RM1],        \
                                           jr1, jr0, ju1, jd1, r.y, T);                                           \
                pq[t.o1] = W1[R0];                                                                                \
            }                                                                                                     \
            /* planes q-3 and q-2 became final in the previous super step */                                     \
            if (!EDGE || q - 3 >= a) writeback(q - 3, QSG_SLOT(Q - 3));                                           \
            if (!EDGE || q - 2 >= a) writeback(q - 2, QSG_SLOT(Q - 2));                                           \
        }                                                                                                         \
        carry = r.z;                                                                                              \
    }

    // the first and last 16 planes of the chunk carry the boundary checks; the
    // interior runs a copy of the same steps without them
    for (int base = a; base < b; base += 16) {
        if (base == a || base + 16 >= b) {
            constexpr bool EDGE = true;
            QSG_SUPER(0)
            QSG_SUPER(1)
            QSG_SUPER(2)
            QSG_SUPER(3)
            QSG_SUPER(4)
            QSG_SUPER(5)
            QSG_SUPER(6)
            QSG_SUPER(7)
        } else {
            constexpr bool EDGE = false;
            QSG_SUPER(0)
            QSG_SUPER(1)
            QSG_SUPER(2)
            QSG_SUPER(3)
            QSG_SUPER(4)
            QSG_SUPER(5)
            QSG_SUPER(6)
            QSG_SUPER(7)
        }
    }
#undef QSG_SUPER

    cp_wait<0>();
    __syncthreads();
    if (active) {
        // planes b-3, b-2 (final) and b-1 (colour-1 sites deferred to the boundary update)
        for (int p = b - 3; p < b; ++p) writeback(p, QSG_SLOT(p - a));
    }
#undef QSG_SLOT
    // arrival at the two chunk boundaries: the second unit to arrive updates them
    __threadfence();
    __syncthreads();
    const int chn = b == Lt ? 0 : ch + 1;  // the chunk after the last is the first
    if (c == 0) {
        int flags = 0;
        if (active) {
            if (atomicAdd(&arrivals[s * astride + ch], 1u) == 1u) flags |= 1;
            if (atomicAdd(&arrivals[s * astride + chn], 1u) == 1u) flags |= 2;
            __threadfence();
        }
        *do_boundary = flags;
    }
    __syncthreads();
    const int flags = *do_boundary;
    if (active && flags) {
        if (flags & 1) boundary_update<ALGO>(g, t, Sg, sJx, sJy, a, T, sweep, (uint32_t)s, k0, k1);
        if (flags & 2) boundary_update<ALGO>(g, t, Sg, sJx, sJy, b == Lt ? 0 : b, T, sweep, (uint32_t)s, k0, k1);
        if (c == 0) {
            if (flags & 1) arrivals[s * astride + ch] = 0u;
            if (flags & 2) arrivals[s * astride + chn] = 0u;
        }
    }
}

// One launch per sweep of one group: P units per block (blocks of P * L^2 / 2
// threads).  Slots [0, S1) run nch chunks of C planes, slots [S1, nslots) nch2
// chunks of C2 <= C planes; the units of the first slots come first, so that
// the shorter units fill the last wave of blocks.
template <int ALGO, int SLOT, int NREG, bool JREG = false>
__global__ void __launch_bounds__(512) __maxnreg__(NREG)
    k_sweep_wavefront(const Group g, const int C, const int nch, const int S1, const int C2, const int nch2,
                      const int P, const uint32_t *sweep_base, const uint32_t sweep_off, const uint32_t k0,
                      const uint32_t k1, unsigned *__restrict__ arrivals) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ int do_boundary[32];
    // absolute sweep index (keys Philox): a device counter plus an offset, so
    // that a captured graph of several sweeps can be replayed at any point
    const uint32_t sweep = (sweep_base ? *sweep_base : 0u) + sweep_off;
    const int L2 = g.L * g.L, tpu = L2 / 2;
    const int u = threadIdx.x / tpu, c = threadIdx.x - u * tpu;
    const int unit = blockIdx.x * P + u;
    const int n1 = S1 * nch;
    const bool active = unit < n1 + (g.nslots - S1) * nch2;
    const bool first = unit < n1;
    const int v = first ? unit : unit - n1;
    const int nu = first ? nch : nch2;
    const int s = active ? (first ? 0 : S1) + v / nu : 0;
    const int ch = active ? v % nu : 0;
    wavefront_unit<ALGO, SLOT, JREG>(g, first ? C : C2, nch2, s, ch, active, c,
                                     smem + (size_t)u * (kRing * SLOT + 2 * L2), &do_boundary[u], sweep, k0, k1,
                                     arrivals);
}

// One launch per sweep of several groups of different sizes (same algorithm):
// a persistent grid pulls units from a queue ordered largest group first;
// every block has 288 threads and SLOT >= the largest L^2, threads beyond a
// unit's L^2 / 2 idle.  queue[0] hands out units, queue[1] counts the blocks
// that have finished; the last one resets both for the next launch.
template <int ALGO, int SLOT, int NREG>
__global__ void __launch_bounds__(288) __maxnreg__(NREG)
    k_sweep_persistent(const Group *__restrict__ groups, const int *__restrict__ order,
                       const int *__restrict__ prefix, const int *__restrict__ chunk, const int ngroups,
                       unsigned *__restrict__ queue, const uint32_t *sweep_base, const uint32_t sweep_off,
                       const uint32_t k0, const uint32_t k1) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ int do_boundary;
    __shared__ int s_unit;
    const uint32_t sweep = (sweep_base ? *sweep_base : 0u) + sweep_off;
    const int total = prefix[ngroups];
    for (;;) {
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(&queue[0], 1u);
        __syncthreads();
        const int unit = s_unit;
        __syncthreads();
        if (unit >= total) break;
        int k = 0;
        while (k + 1 < ngroups && unit >= prefix[k + 1]) ++k;
        const Group g = groups[order[k]];
        const int C = chunk[order[k]], nch = g.Ltau / C;
        const int lu = unit - prefix[k];
        const int s = lu / nch, ch = lu - s * nch;
        const bool active = (int)threadIdx.x < g.L * g.L / 2;
        wavefront_unit<ALGO, SLOT, true>(g, C, nch, s, ch, active, active ? (int)threadIdx.x : 0, smem, &do_boundary, sweep,
                                   k0, k1, g.arrivals);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&queue[1], 1u) == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
        }
    }
}

// Chunk length: a multiple of 16 dividing L_tau; chosen so that there are
// enough units to fill the GPU while chunks stay long (the deferred boundary
// work is about 3 planes per chunk).
int wavefront_chunk(const Group &g, int requested) {
    if (g.Ltau % 16 != 0) return 0;
    if (requested > 0) return (g.Ltau % requested == 0 && requested % 16 == 0) ? requested : 0;
    int C = g.Ltau;
    while (C % 32 == 0 && C / 2 >= 32 && (long long)g.nslots * (g.Ltau / C) < 152LL * 16) C /= 2;
    return C;
}

int g_wavefront_variant = 0;  // see launch_sweep_wavefront

// Work units per block: g.upb rounded down to a power of two with at most 512
// threads, or by default the most that fit 256 threads (up to 16).  Units are
// independent, so the grouping changes no bit.
int wavefront_units_per_block(const Group &g) {
    const int tpu = g.L * g.L / 2;
    int P = 1;
    if (g.upb > 0) {
        while (P * 2 <= g.upb && P * 2 <= 16 && (P * 2) * tpu <= 512) P *= 2;
        return P;
    }
    while ((P * 2) * tpu <= 256 && P * 2 <= 16) P *= 2;
    return P;
}

// Slots whose chunks are a quarter of C (the last `tail` slots), when C allows.
static int tail_slots(const Group &g, int C, int tail) {
    if (tail <= 0 || C < 64 || (C / 4) % 16 != 0) return 0;
    return tail < g.nslots ? tail : g.nslots;
}

template <int ALGO, int SLOT, int NREG, bool JREG = false>
static cudaError_t launch_wf(const Group &g, int C, int tail, const uint32_t *sweep_base, uint32_t sweep,
                             uint64_t seed, unsigned *arrivals, cudaStream_t st) {
    const int nch = g.Ltau / C;
    const int ts = tail_slots(g, C, tail);
    const int C2 = ts > 0 ? C / 4 : C, nch2 = g.Ltau / C2, S1 = g.nslots - ts;
    const int P = wavefront_units_per_block(g);
    const int units = S1 * nch + ts * nch2;
    const int blocks = (units + P - 1) / P;
    const size_t sm = (size_t)P * (kRing * SLOT + 2 * g.L * g.L) * sizeof(uint64_t);
    const int threads = P * (g.L * g.L / 2);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_wavefront<ALGO, SLOT, NREG, JREG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_wavefront<ALGO, SLOT, NREG, JREG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_sweep_wavefront<ALGO, SLOT, NREG, JREG><<<blocks, threads, sm, st>>>(
        g, C, nch, S1, C2, nch2, P, sweep_base, sweep, (uint32_t)seed, (uint32_t)(seed >> 32), arrivals);
    return cudaGetLastError();
}

// Registers are allocated per SM sub-partition (16K each), so a block of 9
// warps (288 threads) fits twice per SM at <= 96 registers; the couplings of
// the thread's sites are held in registers for the whole chunk.  Blocks of
// more than 288 threads get 64.
template <int ALGO, int SLOT>
static cudaError_t launch_wf_slot(const Group &g, int C, int tail, const uint32_t *sb, uint32_t sweep, uint64_t seed,
                                  unsigned *arrivals, cudaStream_t st) {
    const int threads = wavefront_units_per_block(g) * (g.L * g.L / 2);
    if (threads > 288) return launch_wf<ALGO, SLOT, 64, true>(g, C, tail, sb, sweep, seed, arrivals, st);
    return launch_wf<ALGO, SLOT, 96, true>(g, C, tail, sb, sweep, seed, arrivals, st);
}

// Ring planes are padded to the next of a few sizes (exact for L = 8, 12, 16,
// 20, 24, 32).
template <int ALGO>
static cudaError_t launch_wf_algo(const Group &g, int C, int tail, const uint32_t *sb, uint32_t sweep, uint64_t seed,
                                  unsigned *arrivals, cudaStream_t st) {
    const int L2 = g.L * g.L;
    if (L2 <= 64) return launch_wf_slot<ALGO, 64>(g, C, tail, sb, sweep, seed, arrivals, st);
    if (L2 <= 144) return launch_wf_slot<ALGO, 144>(g, C, tail, sb, sweep, seed, arrivals, st);
    if (L2 <= 256) return launch_wf_slot<ALGO, 256>(g, C, tail, sb, sweep, seed, arrivals, st);
    if (L2 <= 400) return launch_wf_slot<ALGO, 400>(g, C, tail, sb, sweep, seed, arrivals, st);
    if (L2 <= 576) return launch_wf_slot<ALGO, 576>(g, C, tail, sb, sweep, seed, arrivals, st);
    return launch_wf_slot<ALGO, 1024>(g, C, tail, sb, sweep, seed, arrivals, st);
}

cudaError_t launch_sweep_wavefront(const Group &g, const uint32_t *sweep_base, uint32_t sweep, uint64_t seed,
                                   unsigned *arrivals, int C, int tail, cudaStream_t st) {
    // one unit per block with the lattice size compiled in (k_sweep_unit.cu)
    // where that kernel exists, unless the generic kernel is asked for
    if (g_wavefront_variant != 2 && sweep_unit_supported(g)) {
        const int ts = tail_slots(g, C, tail);
        // planes per barrier: four by default (the faster form for both
        // algorithms), two as variant 1
        const int pb = g_wavefront_variant == 1 ? 2 : 4;
        return launch_sweep_unit(g, pb, C, ts > 0 ? C / 4 : C, g.nslots - ts, sweep_base, sweep, seed, arrivals, st);
    }
    if (g.algo == 0) return launch_wf_algo<0>(g, C, tail, sweep_base, sweep, seed, arrivals, st);
    return launch_wf_algo<1>(g, C, tail, sweep_base, sweep, seed, arrivals, st);
}

template <int ALGO>
static cudaError_t launch_persistent_algo(const PersistentPlan &pl, const uint32_t *sweep_base, uint32_t sweep,
                                          uint64_t seed, cudaStream_t st) {
    constexpr int SLOT = 576, NREG = 96, THREADS = 288;
    const size_t sm = (size_t)(kRing * SLOT + 2 * SLOT) * sizeof(uint64_t);
    static int blocks_per_sm[2] = {0, 0};
    cudaError_t e;
    if (!blocks_per_sm[ALGO]) {
        e = cudaFuncSetAttribute(k_sweep_persistent<ALGO, SLOT, NREG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sweep_persistent<ALGO, SLOT, NREG>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int n = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_persistent<ALGO, SLOT, NREG>, THREADS, sm);
        if (e != cudaSuccess) return e;
        blocks_per_sm[ALGO] = n > 0 ? n : 1;
    }
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int blocks = sms * blocks_per_sm[ALGO];
    if (blocks > pl.total_units) blocks = pl.total_units;
    // the work queue starts at zero on every launch (the kernel's last block
    // also resets it, but a launch that did not finish must not leave it set)
    e = cudaMemsetAsync(pl.queue, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_sweep_persistent<ALGO, SLOT, NREG><<<blocks, THREADS, sm, st>>>(pl.groups, pl.order, pl.prefix, pl.chunk,
                                                                      pl.ngroups, pl.queue, sweep_base, sweep,
                                                                      (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

cudaError_t launch_sweep_persistent(const PersistentPlan &pl, const uint32_t *sweep_base, uint32_t sweep,
                                    uint64_t seed, cudaStream_t st) {
    if (pl.algo == 0) return launch_persistent_algo<0>(pl, sweep_base, sweep, seed, st);
    return launch_persistent_algo<1>(pl, sweep_base, sweep, seed, st);
}

// ---------------------------------------------------------------------------
// Sweep entry point that allocates nothing.
//
// Its scratch -- the boundary arrival counters of the wavefront kernel and the
// acceptance table -- lives in the two file-scope device arrays below, so a
// caller that cannot allocate device memory only has to pass its own spin and
// coupling buffers.  Every GPU that loads the library keeps these arrays until
// the process exits.
// ---------------------------------------------------------------------------
}  // namespace qsg

#include <cmath>
#include <cstring>
#include <mutex>

#include "qsg.h"

namespace qsg {
namespace {

constexpr int kStaticArrivals = 1 << 20;  // counters: slots x chunks per call (4 MiB)
constexpr int kStaticMaxK = 128;          // ladder positions (16 thresholds each)
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned g_static_arrivals[kStaticArrivals];
__device__ __align__(256) uint32_t g_static_thr[kStaticMaxK * 16];

std::mutex g_static_mutex;
void *g_static_arrivals_ptr[kMaxDevices];
void *g_static_thr_ptr[kMaxDevices];

// Device addresses of the two arrays on device `dev`, which must be current
// (looked up, and the counters cleared, on the first call on that device).
// The addresses are cached per device; they do not survive cudaDeviceReset.
cudaError_t static_scratch(int dev, void **arrivals, void **thr) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_arrivals_ptr[dev]) {
        void *a = nullptr, *t = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_static_arrivals);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&t, g_static_thr);
        if (e != cudaSuccess) return e;
        e = cudaMemset(a, 0, sizeof(unsigned) * kStaticArrivals);
        if (e != cudaSuccess) return e;
        g_static_arrivals_ptr[dev] = a;
        g_static_thr_ptr[dev] = t;
    }
    *arrivals = g_static_arrivals_ptr[dev];
    *thr = g_static_thr_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace qsg

extern "C" qsg_status qsg_sweep_static_scratch(uint64_t *d_spins, const uint64_t *d_Jx, const uint64_t *d_Jy,
                                               const qsg_shape *shape, int32_t group_id, const double *k_ladder,
                                               uint64_t seed, uint32_t first_sweep, int32_t n_sweeps,
                                               void *cuda_stream) {
    using namespace qsg;
    // shape and limits first, so that an oversized shape is reported as such
    // whatever the buffers are
    if (!shape) return QSG_ERR_ARG;
    const qsg_shape &sh = *shape;
    if (sh.L < 2 || sh.L > 32 || (sh.L & 1) || sh.Ltau < 16 || sh.Ltau > 65536 || sh.n_samples < 1 ||
        sh.n_replicas < 1 || sh.n_replicas > 1023 || sh.n_k < 1 ||
        (sh.algo != QSG_METROPOLIS && sh.algo != QSG_HEATBATH) ||
        (sh.boundary != QSG_PBC && sh.boundary != QSG_APBC) || sh.reserved != 0)
        return QSG_ERR_SHAPE;
    Group g;
    memset(&g, 0, sizeof(g));
    g.L = sh.L;
    g.Ltau = sh.Ltau;
    g.W = (sh.n_samples + 63) / 64;
    g.R = sh.n_replicas;
    g.K = sh.n_k;
    g.algo = sh.algo;
    g.boundary = sh.boundary;
    g.gid = group_id;
    g.N = sh.L * sh.L * sh.Ltau;
    g.nslots = g.W * g.R * g.K;
    g.nlag = sh.Ltau / 2 + 1;
    g.n_samples = sh.n_samples;
    g.nwx = (sh.L * sh.L + 63) / 64;
    if ((long long)g.W * g.R * g.K > (1LL << 30)) return QSG_ERR_SHAPE;
    const int C = wavefront_chunk(g, 0);
    if (C == 0) return QSG_ERR_SHAPE;  // L_tau must be a multiple of 16
    // the limits of the static scratch
    if (g.K > kStaticMaxK || (long long)g.nslots * (g.Ltau / C) > kStaticArrivals) return QSG_ERR_WORKSPACE;
    if (!d_spins || !d_Jx || !d_Jy || !k_ladder || n_sweeps < 0 || group_id < 0 || group_id > 255)
        return QSG_ERR_ARG;
    if ((uint64_t)first_sweep + (uint64_t)n_sweeps > 0xFFFFFFFFull) return QSG_ERR_ARG;
    // acceptance table (the definitions of qsg_init_samples), on the stack
    uint32_t table[kStaticMaxK * 16];
    if (!build_accept_tables(k_ladder, g.K, table)) return QSG_ERR_ARG;
    // the scratch is looked up on the current device: the stream must belong to it
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QSG_ERR_CUDA;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return QSG_ERR_ARG;
    if (sdev != dev) return QSG_ERR_ARG;
    void *arr = nullptr, *thr = nullptr;
    if (static_scratch(dev, &arr, &thr) != cudaSuccess) return QSG_ERR_CUDA;
    // the table lives on this function's stack: copy it and wait for the copy
    if (cudaMemcpyAsync(thr, table, sizeof(uint32_t) * 16 * (size_t)g.K, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return QSG_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return QSG_ERR_CUDA;
    // counters start at zero (each sweep leaves them at zero; cleared anyway)
    if (cudaMemsetAsync(arr, 0, sizeof(unsigned) * (size_t)g.nslots * (g.Ltau / C), st) != cudaSuccess)
        return QSG_ERR_CUDA;
    g.S = d_spins;
    g.Jx = const_cast<uint64_t *>(d_Jx);
    g.Jy = const_cast<uint64_t *>(d_Jy);
    g.thr = (uint32_t *)thr;
    for (int it = 0; it < n_sweeps; ++it)
        if (launch_sweep_wavefront(g, nullptr, first_sweep + (uint32_t)it, seed, (unsigned *)arr, C, 0, st) != cudaSuccess)
            return QSG_ERR_CUDA;
    return QSG_OK;
}
