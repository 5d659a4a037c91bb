// k_sweep_unit.cu -- the fused one-pass checkerboard sweep with one work unit
// per thread block and the lattice size known at compile time.
//
// The schedule and every random draw are those of the generic wavefront
// kernel (k_wavefront.cu), so the two produce the same bits: a unit is one
// slot and a chunk of C tau planes streamed through a 16-plane shared-memory
// ring; a thread owns the column pair (x0, x0 + 1) of row y, x0 = 2 xh + (y & 1);
// colour 0 of planes q .. q+PB-1 is updated, then (after one block barrier)
// colour 1 of planes q-1 .. q+PB-2; the colour-1 sites of a chunk's first plane
// and of the plane before it are deferred to whichever of the two adjacent
// units finishes second.
//
// What this form changes, for the integer-ALU budget of a site update:
//  * L is a template parameter: every shared-memory and global offset of the
//    unrolled 16-plane body is a compile-time constant from a few base
//    registers, and the grid has exactly one block per unit (no idle threads,
//    no per-step activity test);
//  * the seven coupling words of a thread's two sites stay in registers for
//    the whole unit (they are read from global memory once, and no shared
//    copy is kept), so a block needs 16 planes of shared memory only;
//  * 72 registers per thread: three blocks of 288 threads per SM at L = 24
//    (four of 200 at L = 20, seven of 128 at L = 16) instead of two;
//  * PB = 4 planes per block barrier (PB = 2 as a variant).  With four
//    planes per step the ring allows a prefetch distance of 10 planes: the
//    planes of step q + 4 are issued after the barrier of step q - 4 and all
//    groups have landed at the barrier of step q.
#include <type_traits>

#include "qsg_launch.h"
#include "qsg_sweep.cuh"

namespace qsg {

namespace {

using namespace sweep;

// Colour-1 sites (x0, pb - 1) and (x0 + 1, pb) around chunk boundary pb, with
// the thread's couplings in registers; spins are read from global memory
// (bypassing L1: the neighbouring unit wrote them).
template <int ALGO, int L>
__device__ __forceinline__ void boundary_sites(const Group &g, int c, uint64_t *Sg, int pb, const Thresh &T,
                                               uint32_t sweep, uint32_t slot, uint32_t k0, uint32_t k1,
                                               uint64_t Jr0, uint64_t Jl0, uint64_t Ju0, uint64_t Jd0, uint64_t Jr1,
                                               uint64_t Ju1, uint64_t Jd1) {
    constexpr int L2 = L * L, half = L / 2;
    const int Lt = g.Ltau;
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;
    const int y = c / half, xh = c % half;
    const int x0 = 2 * xh + (y & 1);
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
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(L * half) + (uint32_t)c, sweep, slot,
                                                 tag), k0, k1);
        Sg[(size_t)p * L2 + n0] =
            update_site<ALGO>(__ldcg(P + n0), __ldcg(P + n1), __ldcg(P + y * L + x0m), __ldcg(P + yp * L + x0),
                              __ldcg(P + ym * L + x0), __ldcg(Pp + n0) ^ fp, __ldcg(Pm + n0), Jr0, Jl0, Ju0, Jd0, r.z,
                              T);
    }
    {
        const int p = pb;  // even plane: x0 + 1 is colour 1
        const uint64_t *P = Sg + (size_t)p * L2;
        const uint64_t *Pp = Sg + (size_t)(p + 1) * L2;
        const uint64_t *Pm = Sg + (size_t)(p == 0 ? Lt - 1 : p - 1) * L2;
        const uint64_t fm = p == 0 ? apbc : 0ull;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(L * half) + (uint32_t)c, sweep, slot,
                                                 tag), k0, k1);
        Sg[(size_t)p * L2 + n1] =
            update_site<ALGO>(__ldcg(P + n1), __ldcg(P + y * L + x1p), __ldcg(P + n0), __ldcg(P + yp * L + x1),
                              __ldcg(P + ym * L + x1), __ldcg(Pp + n1), __ldcg(Pm + n1) ^ fm, Jr1, Jr0, Ju1, Jd1, r.y,
                              T);
    }
}

// 72 registers: three blocks of 288 threads per SM at L = 24, four of 200 at L = 20
// (L = 8, 12, 16 are compiled too: the ragged workloads' smaller lattices)
constexpr int kUnitRegs = 72;

// One launch per sweep of one group, one unit per block (L^2 / 2 threads).
// Slots [0, S1) run nch chunks of C planes, slots [S1, nslots) nch2 chunks of
// C2 = C / 4 planes; the boundary counter at the start of chunk ch of slot s
// is arrivals[s * nch2 + ch].
template <int ALGO, int L, int PB, int NREG = kUnitRegs>
__global__ void __launch_bounds__(L *L / 2) __maxnreg__(NREG)
    k_sweep_unit(const Group g, const int C, const int nch, const int S1, const int C2, const int nch2,
                 const uint32_t *sweep_base, const uint32_t sweep_off, const uint32_t k0, const uint32_t k1,
                 unsigned *__restrict__ arrivals) {
    static_assert(PB == 2 || PB == 4, "two or four planes per barrier");
    constexpr int L2 = L * L, H = L2 / 2, half = L / 2, SLOT = L2;
    constexpr uint32_t qstride = (uint32_t)(L * half);
    extern __shared__ __align__(16) uint64_t ring[];
    __shared__ int do_boundary;
    // absolute sweep index (keys Philox): a device counter plus an offset, so
    // that a captured graph of several sweeps can be replayed at any point
    const uint32_t sweep = (sweep_base ? *sweep_base : 0u) + sweep_off;
    const int unit = blockIdx.x;
    const int n1 = S1 * nch;
    const bool longpart = unit < n1;
    const int v = longpart ? unit : unit - n1;
    const int nu = longpart ? nch : nch2;
    const int s = (longpart ? 0 : S1) + v / nu;
    const int ch = v % nu;
    const int Cu = longpart ? C : C2;
    const int c = threadIdx.x;
    const int Lt = g.Ltau;
    const int a = ch * Cu, b = a + Cu;
    const int w = s / (g.R * g.K), j = s % g.K;
    uint64_t *Sg = g.S + (size_t)s * g.N;
    // thread geometry in the class-split plane: sites with (x + y) even first,
    // then (x + y) odd, each as [y][x / 2]
    const int y = c / half, xh = c % half;
    const int x0 = 2 * xh + (y & 1);
    const int x1 = x0 + 1 == L ? 0 : x0 + 1;
    const int x0m = x0 == 0 ? L - 1 : x0 - 1;
    const int x1p = x1 + 1 == L ? 0 : x1 + 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int o0 = c, o1 = H + y * half + (x1 >> 1);
    const int l0 = H + y * half + (x0m >> 1), u0 = H + yp * half + xh, d0 = H + ym * half + xh;
    const int r1 = y * half + (x1p >> 1), u1 = yp * half + (x1 >> 1), d1 = ym * half + (x1 >> 1);
    const int dA = (y & 1) * H + c, dB = (1 - (y & 1)) * H + c;  // where global words 2c, 2c + 1 land
    // couplings of word-group w at the thread's two sites
    const uint64_t *gJx = g.Jx + (size_t)w * L2, *gJy = g.Jy + (size_t)w * L2;
    const uint64_t Jr0 = __ldg(gJx + y * L + x0), Jl0 = __ldg(gJx + y * L + x0m);
    const uint64_t Ju0 = __ldg(gJy + y * L + x0), Jd0 = __ldg(gJy + ym * L + x0);
    const uint64_t Jr1 = __ldg(gJx + y * L + x1), Ju1 = __ldg(gJy + y * L + x1), Jd1 = __ldg(gJy + ym * L + x1);
    Thresh T;
#pragma unroll
    for (int n = 0; n < 7; ++n) T.t[n] = g.thr[j * 16 + (ALGO == 0 ? n % 3 : 8 + n)];
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;

    // plane p of the chunk lives in ring slot (p - a + 1) & 15; `edge` is false
    // in the interior of the chunk, where every plane issued lies in [a, b)
    auto issue_plane = [&](int p, uint64_t *dst, auto edge) {
        constexpr bool E = decltype(edge)::value;
        if (!E || p <= b) {
            const int gp = !E ? p : (p < 0 ? p + Lt : (p >= Lt ? p - Lt : p));
            const uint64_t *src = Sg + (size_t)gp * L2 + 2 * c;
            cp_async8(dst + dA, src);
            cp_async8(dst + dB, src + 1);
        }
    };
    auto writeback = [&](int p, const uint64_t *src) {
        *reinterpret_cast<ulonglong2 *>(Sg + (size_t)p * L2 + 2 * c) = make_ulonglong2(src[dA], src[dB]);
    };
    // one Philox call feeds the four sites of the thread's 2 x 2 (x, tau)
    // block at tau pair (q, q + 1)
    auto draw = [&](int q) {
        return philox4x32_10(make_uint4((uint32_t)(q >> 1) * qstride + (uint32_t)c, sweep, (uint32_t)s, tag), k0, k1);
    };

    // prologue: planes a-1 .. a+PRE-2 in slots 0 .. PRE-1
    constexpr int PRE = PB == 4 ? 11 : 9;
#pragma unroll
    for (int i = 0; i < PRE; ++i) issue_plane(a - 1 + i, ring + i * SLOT, std::true_type{});
    cp_commit();
    uint4 ra = draw(a), rb = PB == 4 ? draw(a + 2) : make_uint4(0u, 0u, 0u, 0u);
    uint32_t carry = 0;
    cp_wait<0>();
    __syncthreads();
    // own columns of planes q-2 .. q+PB, register index (p - a) & 7
    uint64_t W0[8], W1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) W0[i] = W1[i] = 0;
    W0[7] = ring[o0];  // plane a-1
    W1[7] = ring[o1];
    W0[0] = ring[SLOT + o0];  // plane a
    W1[0] = ring[SLOT + o1];

// ring slot of plane a + p_rel; inside the loop p_rel is taken modulo 16
// (base - a is a multiple of 16), which makes the slot a compile-time constant
#define QSG_SLOT(P_REL) (ring + (((P_REL) + 1) & (kRing - 1)) * SLOT)
#define QSG_OWN(QI)                         \
    {                                       \
        W0[(QI) & 7] = QSG_SLOT(QI)[o0];    \
        W1[(QI) & 7] = QSG_SLOT(QI)[o1];    \
    }
// colour 0 at an even plane (column x0) and at an odd plane (column x0 + 1)
#define QSG_C0_EVEN(QI, U)                                                                                      \
    {                                                                                                           \
        uint64_t *pp = QSG_SLOT(QI);                                                                            \
        constexpr int R = (QI) & 7, RP = ((QI) + 1) & 7, RM = ((QI) + 7) & 7;                                   \
        W0[R] = update_site<ALGO>(W0[R], W1[R], pp[l0], pp[u0], pp[d0], W0[RP],                                 \
                                  W0[RM] ^ (EDGE && base + (QI) == 0 ? apbc : 0ull), Jr0, Jl0, Ju0, Jd0, U, T); \
        pp[o0] = W0[R];                                                                                         \
    }
#define QSG_C0_ODD(QI, U)                                                                                       \
    {                                                                                                           \
        uint64_t *pp = QSG_SLOT(QI);                                                                            \
        constexpr int R = (QI) & 7, RP = ((QI) + 1) & 7, RM = ((QI) + 7) & 7;                                   \
        W1[R] = update_site<ALGO>(W1[R], pp[r1], W0[R], pp[u1], pp[d1],                                         \
                                  W1[RP] ^ (EDGE && base + (QI) == Lt - 1 ? apbc : 0ull), W1[RM], Jr1, Jr0, Ju1, \
                                  Jd1, U, T);                                                                   \
        pp[o1] = W1[R];                                                                                         \
    }
// colour 1 at an odd plane (column x0) and at an even plane (column x0 + 1);
// never a chunk-boundary plane, so no wrap sign
#define QSG_C1_ODD(QI, U)                                                                                       \
    {                                                                                                           \
        uint64_t *pp = QSG_SLOT(QI);                                                                            \
        constexpr int R = (QI) & 7, RP = ((QI) + 1) & 7, RM = ((QI) + 7) & 7;                                   \
        W0[R] = update_site<ALGO>(W0[R], W1[R], pp[l0], pp[u0], pp[d0], W0[RP], W0[RM], Jr0, Jl0, Ju0, Jd0, U, T); \
        pp[o0] = W0[R];                                                                                         \
    }
#define QSG_C1_EVEN(QI, U)                                                                                      \
    {                                                                                                           \
        uint64_t *pp = QSG_SLOT(QI);                                                                            \
        constexpr int R = (QI) & 7, RP = ((QI) + 1) & 7, RM = ((QI) + 7) & 7;                                   \
        W1[R] = update_site<ALGO>(W1[R], pp[r1], W0[R], pp[u1], pp[d1], W1[RP], W1[RM], Jr1, Jr0, Ju1, Jd1, U, T); \
        pp[o1] = W1[R];                                                                                         \
    }
// two planes per barrier: issue planes q+8, q+9 before the barrier, which
// waits for everything but the last two groups (planes <= q+5)
#define QSG_STEP2(MM)                                                                                           \
    {                                                                                                           \
        constexpr int Q = 2 * (MM);                                                                             \
        const int q = base + Q;                                                                                 \
        QSG_OWN(Q + 1)                                                                                          \
        QSG_OWN(Q + 2)                                                                                          \
        issue_plane(q + 8, QSG_SLOT(Q + 8), std::integral_constant<bool, EDGE>{});                              \
        issue_plane(q + 9, QSG_SLOT(Q + 9), std::integral_constant<bool, EDGE>{});                              \
        cp_commit();                                                                                            \
        const uint4 r = ra;                                                                                     \
        QSG_C0_EVEN(Q, r.x)                                                                                     \
        QSG_C0_ODD(Q + 1, r.w)                                                                                  \
        cp_wait<2>();                                                                                           \
        __syncthreads();                                                                                        \
        if (!EDGE || q >= a + 2) {                                                                              \
            QSG_C1_ODD(Q - 1, carry)                                                                            \
            QSG_C1_EVEN(Q, r.y)                                                                                 \
        }                                                                                                       \
        ra = draw(q + 2);                                                                                       \
        if (!EDGE || q - 3 >= a) writeback(q - 3, QSG_SLOT(Q - 3));                                             \
        if (!EDGE || q - 2 >= a) writeback(q - 2, QSG_SLOT(Q - 2));                                             \
        carry = r.z;                                                                                            \
    }
// four planes per barrier: the barrier waits for every group; planes q+10 ..
// q+13 are issued after it, once planes q-5 .. q-2 have been written back.
// The next step's random numbers are drawn after the colour-1 updates, when
// this step's are dead (fewer live registers at 72)
#define QSG_STEP4(MM)                                                                                           \
    {                                                                                                           \
        constexpr int Q = 4 * (MM);                                                                             \
        const int q = base + Q;                                                                                 \
        QSG_OWN(Q + 1)                                                                                          \
        QSG_OWN(Q + 2)                                                                                          \
        QSG_OWN(Q + 3)                                                                                          \
        QSG_OWN(Q + 4)                                                                                          \
        const uint4 rq0 = ra, rq1 = rb;                                                                         \
        QSG_C0_EVEN(Q, rq0.x)                                                                                   \
        QSG_C0_ODD(Q + 1, rq0.w)                                                                                \
        QSG_C0_EVEN(Q + 2, rq1.x)                                                                               \
        QSG_C0_ODD(Q + 3, rq1.w)                                                                                \
        cp_wait<0>();                                                                                           \
        __syncthreads();                                                                                        \
        if (!EDGE || q >= a + 4) {                                                                              \
            QSG_C1_ODD(Q - 1, carry)                                                                            \
            QSG_C1_EVEN(Q, rq0.y)                                                                               \
        }                                                                                                       \
        QSG_C1_ODD(Q + 1, rq0.z)                                                                                \
        QSG_C1_EVEN(Q + 2, rq1.y)                                                                               \
        ra = draw(q + 4);                                                                                       \
        rb = draw(q + 6);                                                                                       \
        if (!EDGE || q - 5 >= a) writeback(q - 5, QSG_SLOT(Q - 5));                                             \
        if (!EDGE || q - 4 >= a) writeback(q - 4, QSG_SLOT(Q - 4));                                             \
        if (!EDGE || q - 3 >= a) writeback(q - 3, QSG_SLOT(Q - 3));                                             \
        if (!EDGE || q - 2 >= a) writeback(q - 2, QSG_SLOT(Q - 2));                                             \
        issue_plane(q + 10, QSG_SLOT(Q + 10), std::integral_constant<bool, EDGE>{});                            \
        issue_plane(q + 11, QSG_SLOT(Q + 11), std::integral_constant<bool, EDGE>{});                            \
        issue_plane(q + 12, QSG_SLOT(Q + 12), std::integral_constant<bool, EDGE>{});                            \
        issue_plane(q + 13, QSG_SLOT(Q + 13), std::integral_constant<bool, EDGE>{});                            \
        cp_commit();                                                                                            \
        carry = rq1.z;                                                                                          \
    }

    // the first and last 16 planes of the chunk carry the boundary checks; the
    // interior runs a copy of the same steps without them
    for (int base = a; base < b; base += 16) {
        if (base == a || base + 16 >= b) {
            constexpr bool EDGE = true;
            if (PB == 4) {
                QSG_STEP4(0) QSG_STEP4(1) QSG_STEP4(2) QSG_STEP4(3)
            } else {
                QSG_STEP2(0) QSG_STEP2(1) QSG_STEP2(2) QSG_STEP2(3) QSG_STEP2(4) QSG_STEP2(5) QSG_STEP2(6) QSG_STEP2(7)
            }
        } else {
            constexpr bool EDGE = false;
            if (PB == 4) {
                QSG_STEP4(0) QSG_STEP4(1) QSG_STEP4(2) QSG_STEP4(3)
            } else {
                QSG_STEP2(0) QSG_STEP2(1) QSG_STEP2(2) QSG_STEP2(3) QSG_STEP2(4) QSG_STEP2(5) QSG_STEP2(6) QSG_STEP2(7)
            }
        }
    }
#undef QSG_STEP4
#undef QSG_STEP2
#undef QSG_C1_EVEN
#undef QSG_C1_ODD
#undef QSG_C0_ODD
#undef QSG_C0_EVEN
#undef QSG_OWN

    cp_wait<0>();
    __syncthreads();
    // the last planes: final ones, and b-1 (its colour-1 sites are deferred)
    for (int p = b - (PB == 4 ? 5 : 3); p < b; ++p) writeback(p, QSG_SLOT(p - a));
#undef QSG_SLOT
    // arrival at the two chunk boundaries: the second unit to arrive updates them
    __threadfence();
    __syncthreads();
    const int chn = b == Lt ? 0 : ch + 1;  // the chunk after the last is the first
    if (c == 0) {
        int flags = 0;
        if (atomicAdd(&arrivals[s * nch2 + ch], 1u) == 1u) flags |= 1;
        if (atomicAdd(&arrivals[s * nch2 + chn], 1u) == 1u) flags |= 2;
        __threadfence();
        do_boundary = flags;
    }
    __syncthreads();
    const int flags = do_boundary;
    if (flags) {
        if (flags & 1)
            boundary_sites<ALGO, L>(g, c, Sg, a, T, sweep, (uint32_t)s, k0, k1, Jr0, Jl0, Ju0, Jd0, Jr1, Ju1, Jd1);
        if (flags & 2)
            boundary_sites<ALGO, L>(g, c, Sg, b == Lt ? 0 : b, T, sweep, (uint32_t)s, k0, k1, Jr0, Jl0, Ju0, Jd0, Jr1,
                                    Ju1, Jd1);
        if (c == 0) {
            if (flags & 1) arrivals[s * nch2 + ch] = 0u;
            if (flags & 2) arrivals[s * nch2 + chn] = 0u;
        }
    }
}

template <int ALGO, int L, int PB>
cudaError_t launch_unit(const Group &g, int C, int C2, int S1, const uint32_t *sweep_base, uint32_t sweep,
                        uint64_t seed, unsigned *arrivals, cudaStream_t st) {
    const int nch = g.Ltau / C, nch2 = g.Ltau / C2;
    const int units = S1 * nch + (g.nslots - S1) * nch2;
    const size_t sm = (size_t)kRing * L * L * sizeof(uint64_t);
    auto kern = k_sweep_unit<ALGO, L, PB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    count_launches(1);
    kern<<<units, L * L / 2, sm, st>>>(g, C, nch, S1, C2, nch2, sweep_base, sweep, (uint32_t)seed,
                                       (uint32_t)(seed >> 32), arrivals);
    return cudaGetLastError();
}

template <int ALGO, int PB>
cudaError_t launch_unit_L(const Group &g, int C, int C2, int S1, const uint32_t *sb, uint32_t sweep, uint64_t seed,
                          unsigned *arrivals, cudaStream_t st) {
    switch (g.L) {
        case 8: return launch_unit<ALGO, 8, PB>(g, C, C2, S1, sb, sweep, seed, arrivals, st);
        case 12: return launch_unit<ALGO, 12, PB>(g, C, C2, S1, sb, sweep, seed, arrivals, st);
        case 16: return launch_unit<ALGO, 16, PB>(g, C, C2, S1, sb, sweep, seed, arrivals, st);
        case 20: return launch_unit<ALGO, 20, PB>(g, C, C2, S1, sb, sweep, seed, arrivals, st);
        default: return launch_unit<ALGO, 24, PB>(g, C, C2, S1, sb, sweep, seed, arrivals, st);
    }
}

}  // namespace

bool sweep_unit_supported(const Group &g) {
    return (g.L == 8 || g.L == 12 || g.L == 16 || g.L == 20 || g.L == 24) && g.Ltau % 16 == 0;
}

cudaError_t launch_sweep_unit(const Group &g, int planes_per_barrier, int C, int C2, int S1,
                              const uint32_t *sweep_base, uint32_t sweep, uint64_t seed, unsigned *arrivals,
                              cudaStream_t st) {
    if (!sweep_unit_supported(g) || C < 16 || C2 < 16 || g.Ltau % C || g.Ltau % C2 || C % 16 || C2 % 16)
        return cudaErrorInvalidValue;
    if (g.algo == 0)
        return planes_per_barrier == 2 ? launch_unit_L<0, 2>(g, C, C2, S1, sweep_base, sweep, seed, arrivals, st)
                                       : launch_unit_L<0, 4>(g, C, C2, S1, sweep_base, sweep, seed, arrivals, st);
    return planes_per_barrier == 2 ? launch_unit_L<1, 2>(g, C, C2, S1, sweep_base, sweep, seed, arrivals, st)
                                   : launch_unit_L<1, 4>(g, C, C2, S1, sweep_base, sweep, seed, arrivals, st);
}

}  // namespace qsg
