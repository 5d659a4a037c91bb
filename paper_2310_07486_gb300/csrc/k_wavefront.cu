// k_wavefront.cu -- one full checkerboard sweep (colour 0 then colour 1) in a
// single pass over HBM: every spin word is read once and written once.
//
// A work unit is one slot and one chunk of C consecutive tau planes [a, b).
// The unit streams its planes through a shared-memory ring filled by cp.async
// kPrefetch planes ahead.  At step tau it updates the colour-0 sites of plane
// tau (their colour-1 neighbours in planes tau-1, tau, tau+1 are still the old
// ones) and then the colour-1 sites of plane tau-1 (their colour-0 neighbours in
// planes tau-2, tau-1, tau are already new), which is exactly the order of a
// colour-0 half sweep followed by a colour-1 half sweep.
//
// The colour-1 sites of the first plane of a chunk need the new colour 0 of the
// previous chunk's last plane, and vice versa, so the colour-1 sites of planes
// a-1 and a are deferred: whichever of the two units adjacent to the boundary
// finishes second updates them (an atomic arrival counter, no waiting).
//
// Thread layout: a thread owns two neighbouring columns (x0, x0+1) of one row,
// with pairs starting at x = y & 1, so that at step tau the active column is
// x0 + (tau & 1) for every thread of the block (no divergence), and one Philox
// call per 2 x 2 (x, tau) block serves the four updates of that block.
#include "qsg_launch.h"

namespace qsg {

namespace {

constexpr int kRing = 8;                  // planes held in shared memory
constexpr int kPrefetch = kRing - 3;      // planes loaded ahead of the step

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One site update on multispin words.  Terms: nr/nl/nu/nd spatial neighbours
// with couplings jr/jl/ju/jd, ntp/ntm time neighbours (APBC sign folded in).
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

template <int ALGO>
__device__ __forceinline__ uint64_t update_site(uint64_t c, uint64_t nr, uint64_t nl, uint64_t nu, uint64_t nd,
                                                uint64_t ntp, uint64_t ntm, uint64_t jr, uint64_t jl, uint64_t ju,
                                                uint64_t jd, uint32_t u, const Thresh &T) {
    uint64_t b0, b1, b2;
    uint32_t m0, m1, m2;
    threshold_masks<ALGO>(u, T, m0, m1, m2);
    const uint64_t M0 = widen(m0), M1 = widen(m1), M2 = widen(m2);
    if (ALGO == 0) {
        count6(c ^ nr ^ jr, c ^ nl ^ jl, c ^ nu ^ ju, c ^ nd ^ jd, c ^ ntp, c ^ ntm, b0, b1, b2);
    } else {
        count6(nr ^ jr, nl ^ jl, nu ^ ju, nd ^ jd, ntp, ntm, b0, b1, b2);
    }
    const uint64_t e0 = b0 | ~M0;
    const uint64_t e1 = (b1 & ~M1) | (~(b1 ^ M1) & e0);
    const uint64_t ge = (b2 & ~M2) | (~(b2 ^ M2) & e1);
    return ALGO == 0 ? (c ^ ge) : ge;
}

struct Thr {
    int own0, own1;                  // plane offsets of the two owned columns
    int offl0, offu0, offd0;         // neighbours of column x0 (left, up, down)
    int offr1, offu1, offd1;         // neighbours of column x0+1 (right, up, down)
    uint32_t qrow;                   // Philox block index within a tau pair
};

// Couplings of the bonds around one site, read from the unit's J planes in
// shared memory (Jx at a site = bond to x+1, Jy at a site = bond to y+1).
struct Bonds {
    uint64_t r, l, u, d;
};
__device__ __forceinline__ Bonds bonds0(const uint64_t *Jx, const uint64_t *Jy, const Thr &t) {
    return Bonds{Jx[t.own0], Jx[t.offl0], Jy[t.own0], Jy[t.offd0]};
}
__device__ __forceinline__ Bonds bonds1(const uint64_t *Jx, const uint64_t *Jy, const Thr &t) {
    return Bonds{Jx[t.own1], Jx[t.own0], Jy[t.own1], Jy[t.offd1]};
}

__device__ __forceinline__ Thr make_thr(const Group &g, int c) {
    const int L = g.L, half = L / 2;
    const int y = c / half, xh = c % half;
    const int x0 = 2 * xh + (y & 1);
    const int x1 = x0 + 1 == L ? 0 : x0 + 1;
    const int x0m = x0 == 0 ? L - 1 : x0 - 1;
    const int x1p = x1 + 1 == L ? 0 : x1 + 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    Thr t;
    t.own0 = y * L + x0;
    t.own1 = y * L + x1;
    t.offl0 = y * L + x0m;
    t.offu0 = yp * L + x0;
    t.offd0 = ym * L + x0;
    t.offr1 = y * L + x1p;
    t.offu1 = yp * L + x1;
    t.offd1 = ym * L + x1;
    t.qrow = (uint32_t)(y * half + xh);
    return t;
}

// Colour-1 sites of the two planes around chunk boundary pb: (x0, pb-1) and
// (x0+1, pb); all their neighbours are final colour-0 sites.  Reads bypass L1
// because the neighbouring unit wrote them.
template <int ALGO>
__device__ __forceinline__ void boundary_update(const Group &g, const Thr &t, uint64_t *Sg, const uint64_t *Jx,
                                                const uint64_t *Jy, int pb, const Thresh &T, uint32_t sweep,
                                                uint32_t slot, uint32_t k0, uint32_t k1) {
    const int L2 = g.L * g.L, Lt = g.Ltau, half = g.L / 2;
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;
    {
        const int p = pb == 0 ? Lt - 1 : pb - 1;  // odd plane
        const uint64_t *P = Sg + (size_t)p * L2;
        const uint64_t *Pp = Sg + (size_t)(p + 1 == Lt ? 0 : p + 1) * L2;
        const uint64_t *Pm = Sg + (size_t)(p - 1) * L2;
        const uint64_t fp = p == Lt - 1 ? apbc : 0ull;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(g.L * half) + t.qrow, sweep, slot, tag), k0, k1);
        const Bonds j = bonds0(Jx, Jy, t);
        const uint64_t v = update_site<ALGO>(__ldcg(P + t.own0), __ldcg(P + t.own1), __ldcg(P + t.offl0),
                                             __ldcg(P + t.offu0), __ldcg(P + t.offd0), __ldcg(Pp + t.own0) ^ fp,
                                             __ldcg(Pm + t.own0), j.r, j.l, j.u, j.d, r.z, T);
        Sg[(size_t)p * L2 + t.own0] = v;
    }
    {
        const int p = pb;  // even plane
        const uint64_t *P = Sg + (size_t)p * L2;
        const uint64_t *Pp = Sg + (size_t)(p + 1) * L2;
        const uint64_t *Pm = Sg + (size_t)(p == 0 ? Lt - 1 : p - 1) * L2;
        const uint64_t fm = p == 0 ? apbc : 0ull;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(g.L * half) + t.qrow, sweep, slot, tag), k0, k1);
        const Bonds j = bonds1(Jx, Jy, t);
        const uint64_t v = update_site<ALGO>(__ldcg(P + t.own1), __ldcg(P + t.offr1), __ldcg(P + t.own0),
                                             __ldcg(P + t.offu1), __ldcg(P + t.offd1), __ldcg(Pp + t.own1),
                                             __ldcg(Pm + t.own1) ^ fm, j.r, j.l, j.u, j.d, r.y, T);
        Sg[(size_t)p * L2 + t.own1] = v;
    }
}

}  // namespace

template <int ALGO, int NS, int NREG>
__global__ void __launch_bounds__(512) __maxnreg__(NREG)
    k_sweep_wavefront(const Group g, const int C, const int nch, const int P, const uint32_t sweep, const uint32_t k0,
                      const uint32_t k1, unsigned *__restrict__ arrivals) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ int do_boundary[32];
    const int L = g.L, L2 = L * L, Lt = g.Ltau, half = L / 2;
    const int tpu = L2 / 2;
    const int u = threadIdx.x / tpu, c = threadIdx.x - u * tpu;
    const int unit = blockIdx.x * P + u;
    const int RN = g.R / NS;                         // slot sets per (w, j)
    const bool active = unit < g.W * RN * g.K * nch;
    const int set = active ? unit / nch : 0;
    const int ch = active ? unit - set * nch : 0;
    const int a = ch * C, b = a + C;
    const int j = set % g.K, rn = (set / g.K) % RN, w = set / (g.K * RN);
    const int s0 = (w * g.R + rn * NS) * g.K + j;    // slot of the first replica; the others follow at +K
    uint64_t *ring = smem + (size_t)u * (NS * kRing + 2) * L2;
    uint64_t *sJx = ring + NS * kRing * L2, *sJy = sJx + L2;
    const Thr t = make_thr(g, c);
    {
        const uint64_t *gJx = g.Jx + (size_t)w * L2, *gJy = g.Jy + (size_t)w * L2;
        for (int i = c; i < L2; i += tpu) {
            sJx[i] = gJx[i];
            sJy[i] = gJy[i];
        }
    }
    Thresh T;
#pragma unroll
    for (int n = 0; n < 7; ++n) T.t[n] = g.thr[j * 16 + (ALGO == 0 ? n % 3 : 8 + n)];
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint32_t qstride = (uint32_t)(L * half);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;

    auto slot_of = [&](int k, int p) -> uint64_t * {
        return ring + (k * kRing + ((p - a + 2) & (kRing - 1))) * L2;
    };
    auto gplane = [&](int k, int p) -> uint64_t * {
        return g.S + (size_t)(s0 + k * g.K) * g.N + (size_t)p * L2;
    };
    auto issue = [&](int p) {
        if (active && p <= b) {
            const int gp = p < 0 ? p + Lt : (p >= Lt ? p - Lt : p);
#pragma unroll
            for (int k = 0; k < NS; ++k) cp_async16(slot_of(k, p) + 2 * c, gplane(k, gp) + 2 * c);
        }
        cp_commit();
    };

#pragma unroll
    for (int i = 0; i <= kPrefetch; ++i) issue(a - 1 + i);

    // own columns x0, x0+1 of every slot at planes tau-2 .. tau+1, index =
    // plane & 3 (a is a multiple of 4: plane a-1 at index 3, plane a at 0)
    uint64_t W0[NS][4], W1[NS][4];
    uint32_t o_y[NS], o_w[NS], carry[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        W0[k][1] = W0[k][2] = W1[k][1] = W1[k][2] = 0;
        o_y[k] = o_w[k] = carry[k] = 0;
    }
    cp_wait<kPrefetch - 2>();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        W0[k][3] = slot_of(k, a - 1)[t.own0];
        W1[k][3] = slot_of(k, a - 1)[t.own1];
        W0[k][0] = slot_of(k, a)[t.own0];
        W1[k][0] = slot_of(k, a)[t.own1];
    }

    // One step; I = tau & 3 is a compile-time constant in the unrolled loop.
#define QSG_WF_STEP(I)                                                                                            \
    {                                                                                                             \
        const int tau = base + (I);                                                                               \
        constexpr int IP1 = ((I) + 1) & 3, IM1 = ((I) + 3) & 3, IM2 = ((I) + 2) & 3;                             \
        cp_wait<kPrefetch - 2>();                                                                                 \
        __syncthreads();                                                                                          \
        _Pragma("unroll") for (int k = 0; k < NS; ++k) {                                                          \
            const uint64_t *nxt = slot_of(k, tau + 1);                                                            \
            W0[k][IP1] = nxt[t.own0];                                                                             \
            W1[k][IP1] = nxt[t.own1];                                                                             \
        }                                                                                                         \
        issue(tau + kPrefetch);                                                                                   \
        if (active) {                                                                                             \
            const uint64_t fp = tau == Lt - 1 ? apbc : 0ull, fm = tau == 0 ? apbc : 0ull;                         \
            const bool ph2 = tau >= a + 2;                                                                        \
            if (((I) & 1) == 0) {                                                                                 \
                const Bonds jb = bonds0(sJx, sJy, t);                                                             \
                _Pragma("unroll") for (int k = 0; k < NS; ++k) {                                                  \
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)(tau >> 1) * qstride + t.qrow, sweep,      \
                                                             (uint32_t)(s0 + k * g.K), tag), k0, k1);             \
                    uint64_t *pl = slot_of(k, tau);                                                               \
                    W0[k][I] = update_site<ALGO>(W0[k][I], W1[k][I], pl[t.offl0], pl[t.offu0], pl[t.offd0],       \
                                                 W0[k][IP1] ^ fp, W0[k][IM1] ^ fm, jb.r, jb.l, jb.u, jb.d, r.x, T); \
                    pl[t.own0] = W0[k][I];                                                                        \
                    if (ph2) {                                                                                    \
                        uint64_t *pm = slot_of(k, tau - 1);                                                       \
                        W0[k][IM1] = update_site<ALGO>(W0[k][IM1], W1[k][IM1], pm[t.offl0], pm[t.offu0],          \
                                                       pm[t.offd0], W0[k][I], W0[k][IM2], jb.r, jb.l, jb.u, jb.d, \
                                                       carry[k], T);                                              \
                        pm[t.own0] = W0[k][IM1];                                                                  \
                    }                                                                                             \
                    carry[k] = r.z;                                                                               \
                    o_y[k] = r.y;                                                                                 \
                    o_w[k] = r.w;                                                                                 \
                }                                                                                                 \
            } else {                                                                                              \
                const Bonds jb = bonds1(sJx, sJy, t);                                                             \
                _Pragma("unroll") for (int k = 0; k < NS; ++k) {                                                  \
                    uint64_t *pl = slot_of(k, tau);                                                               \
                    W1[k][I] = update_site<ALGO>(W1[k][I], pl[t.offr1], W0[k][I], pl[t.offu1], pl[t.offd1],       \
                                                 W1[k][IP1] ^ fp, W1[k][IM1] ^ fm, jb.r, jb.l, jb.u, jb.d,        \
                                                 o_w[k], T);                                                      \
                    pl[t.own1] = W1[k][I];                                                                        \
                    if (ph2) {                                                                                    \
                        uint64_t *pm = slot_of(k, tau - 1);                                                       \
                        W1[k][IM1] = update_site<ALGO>(W1[k][IM1], pm[t.offr1], W0[k][IM1], pm[t.offu1],          \
                                                       pm[t.offd1], W1[k][I], W1[k][IM2], jb.r, jb.l, jb.u, jb.d, \
                                                       o_y[k], T);                                                \
                        pm[t.own1] = W1[k][IM1];                                                                  \
                    }                                                                                             \
                }                                                                                                 \
            }                                                                                                     \
            if (tau - 2 >= a) {                                                                                   \
                _Pragma("unroll") for (int k = 0; k < NS; ++k) {                                                  \
                    *reinterpret_cast<ulonglong2 *>(gplane(k, tau - 2) + 2 * c) =                                 \
                        *reinterpret_cast<const ulonglong2 *>(slot_of(k, tau - 2) + 2 * c);                       \
                }                                                                                                 \
            }                                                                                                     \
        }                                                                                                         \
    }

    for (int base = a; base < b; base += 4) {
        QSG_WF_STEP(0)
        QSG_WF_STEP(1)
        QSG_WF_STEP(2)
        QSG_WF_STEP(3)
    }
#undef QSG_WF_STEP

    cp_wait<0>();
    __syncthreads();
    if (active) {
        for (int p = b - 2; p < b; ++p) {
#pragma unroll
            for (int k = 0; k < NS; ++k)
                *reinterpret_cast<ulonglong2 *>(gplane(k, p) + 2 * c) =
                    *reinterpret_cast<const ulonglong2 *>(slot_of(k, p) + 2 * c);
        }
    }
    // arrival at the two chunk boundaries: the second unit to arrive updates them
    __threadfence();
    __syncthreads();
    const int chn = ch + 1 == nch ? 0 : ch + 1;
    if (c == 0) {
        int flags = 0;
        if (active) {
            if (atomicAdd(&arrivals[s0 * nch + ch], 1u) == 1u) flags |= 1;
            if (atomicAdd(&arrivals[s0 * nch + chn], 1u) == 1u) flags |= 2;
            __threadfence();
        }
        do_boundary[u] = flags;
    }
    __syncthreads();
    const int flags = do_boundary[u];
    if (active && flags) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            uint64_t *Sg = g.S + (size_t)(s0 + k * g.K) * g.N;
            if (flags & 1) boundary_update<ALGO>(g, t, Sg, sJx, sJy, a, T, sweep, (uint32_t)(s0 + k * g.K), k0, k1);
            if (flags & 2)
                boundary_update<ALGO>(g, t, Sg, sJx, sJy, b == Lt ? 0 : b, T, sweep, (uint32_t)(s0 + k * g.K), k0, k1);
        }
        if (c == 0) {
            if (flags & 1) arrivals[s0 * nch + ch] = 0u;
            if (flags & 2) arrivals[s0 * nch + chn] = 0u;
        }
    }
}

// Chunk length: a multiple of 4 dividing L_tau; chosen so that there are
// enough units to fill the GPU while chunks stay long (the deferred boundary
// work is about 3 planes per chunk).
int wavefront_chunk(const Group &g, int requested) {
    if (g.Ltau % 4 != 0 || g.Ltau < 8) return 0;
    if (requested > 0) return (g.Ltau % requested == 0 && requested % 4 == 0 && requested >= 4) ? requested : 0;
    int C = g.Ltau;
    while (C % 8 == 0 && C / 2 >= 32 && (long long)g.nslots * (g.Ltau / C) < 152LL * 16) C /= 2;
    return C;
}

size_t wavefront_smem_bytes(const Group &g, int P, int NS) {
    return (size_t)P * (NS * kRing + 2) * g.L * g.L * sizeof(uint64_t);
}

int g_wavefront_variant = 0;  // see launch_wf_algo

int wavefront_units_per_block(const Group &g) {
    const int tpu = g.L * g.L / 2;
    int P = 1;
    while ((P * 2) * tpu <= 256 && P * 2 <= 16) P *= 2;
    return P;
}

template <int ALGO, int NS, int NREG>
static cudaError_t launch_wf(const Group &g, int C, uint32_t sweep, uint64_t seed, unsigned *arrivals, cudaStream_t st) {
    const int nch = g.Ltau / C;
    const int P = wavefront_units_per_block(g);
    const int units = g.W * (g.R / NS) * g.K * nch;
    const int blocks = (units + P - 1) / P;
    const size_t sm = wavefront_smem_bytes(g, P, NS);
    const int threads = P * (g.L * g.L / 2);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_wavefront<ALGO, NS, NREG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_wavefront<ALGO, NS, NREG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_sweep_wavefront<ALGO, NS, NREG><<<blocks, threads, sm, st>>>(g, C, nch, P, sweep, (uint32_t)seed,
                                                                   (uint32_t)(seed >> 32), arrivals);
    return cudaGetLastError();
}

// Variants (process-wide option): 0 = one slot per thread, 96 registers;
// 1 = two replicas per thread (same couplings and thresholds), 128 registers;
// 2 = one slot per thread, 72 registers.  Blocks of more than 288 threads use
// a 64-register budget with one slot, whatever the variant.
template <int ALGO>
static cudaError_t launch_wf_algo(const Group &g, int C, uint32_t sweep, uint64_t seed, unsigned *arrivals,
                                  cudaStream_t st) {
    const int threads = wavefront_units_per_block(g) * (g.L * g.L / 2);
    if (threads > 288) return launch_wf<ALGO, 1, 64>(g, C, sweep, seed, arrivals, st);
    if (g_wavefront_variant == 1 && g.R % 2 == 0) return launch_wf<ALGO, 2, 128>(g, C, sweep, seed, arrivals, st);
    if (g_wavefront_variant == 2) return launch_wf<ALGO, 1, 72>(g, C, sweep, seed, arrivals, st);
    return launch_wf<ALGO, 1, 96>(g, C, sweep, seed, arrivals, st);
}

cudaError_t launch_sweep_wavefront(const Group &g, uint32_t sweep, uint64_t seed, unsigned *arrivals, int C,
                                   cudaStream_t st) {
    if (g.algo == 0) return launch_wf_algo<0>(g, C, sweep, seed, arrivals, st);
    return launch_wf_algo<1>(g, C, sweep, seed, arrivals, st);
}

}  // namespace qsg
