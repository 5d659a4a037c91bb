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
template <int ALGO>
__device__ __forceinline__ uint64_t update_site(uint64_t c, uint64_t nr, uint64_t nl, uint64_t nu, uint64_t nd,
                                                uint64_t ntp, uint64_t ntm, uint64_t jr, uint64_t jl, uint64_t ju,
                                                uint64_t jd, uint32_t u, const uint32_t *T) {
    uint64_t b0, b1, b2;
    if (ALGO == 0) {
        count6(c ^ nr ^ jr, c ^ nl ^ jl, c ^ nu ^ ju, c ^ nd ^ jd, c ^ ntp, c ^ ntm, b0, b1, b2);
        return c ^ ge_scalar(b0, b1, b2, 3u - count_above3(u, T));
    } else {
        count6(nr ^ jr, nl ^ jl, nu ^ ju, nd ^ jd, ntp, ntm, b0, b1, b2);
        return ge_scalar(b0, b1, b2, count_above7(u, T));
    }
}

struct Thr {
    int own0, own1;                  // plane offsets of the two owned columns
    int offl0, offu0, offd0;         // neighbours of column x0 (left, up, down)
    int offr1, offu1, offd1;         // neighbours of column x0+1 (right, up, down)
    uint64_t jr0, jl0, ju0, jd0;     // couplings around x0 (right = bond x0 -> x0+1)
    uint64_t jr1, ju1, jd1;          // couplings around x0+1 (left is jr0)
    uint32_t qrow;                   // Philox block index within a tau pair
};

__device__ __forceinline__ Thr make_thr(const Group &g, int c, int w) {
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
    const uint64_t *Jx = g.Jx + (size_t)w * L * L, *Jy = g.Jy + (size_t)w * L * L;
    t.jr0 = Jx[y * L + x0];
    t.jl0 = Jx[y * L + x0m];
    t.ju0 = Jy[y * L + x0];
    t.jd0 = Jy[ym * L + x0];
    t.jr1 = Jx[y * L + x1];
    t.ju1 = Jy[y * L + x1];
    t.jd1 = Jy[ym * L + x1];
    t.qrow = (uint32_t)(y * half + xh);
    return t;
}

// Colour-1 sites of the two planes around chunk boundary pb: (x0, pb-1) and
// (x0+1, pb); all their neighbours are final colour-0 sites.  Reads bypass L1
// because the neighbouring unit wrote them.
template <int ALGO>
__device__ void boundary_update(const Group &g, const Thr &t, uint64_t *Sg, int pb, const uint32_t *T, uint32_t sweep,
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
        const uint64_t v = update_site<ALGO>(__ldcg(P + t.own0), __ldcg(P + t.own1), __ldcg(P + t.offl0),
                                             __ldcg(P + t.offu0), __ldcg(P + t.offd0), __ldcg(Pp + t.own0) ^ fp,
                                             __ldcg(Pm + t.own0), t.jr0, t.jl0, t.ju0, t.jd0, r.z, T);
        Sg[(size_t)p * L2 + t.own0] = v;
    }
    {
        const int p = pb;  // even plane
        const uint64_t *P = Sg + (size_t)p * L2;
        const uint64_t *Pp = Sg + (size_t)(p + 1) * L2;
        const uint64_t *Pm = Sg + (size_t)(p == 0 ? Lt - 1 : p - 1) * L2;
        const uint64_t fm = p == 0 ? apbc : 0ull;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(p >> 1) * (uint32_t)(g.L * half) + t.qrow, sweep, slot, tag), k0, k1);
        const uint64_t v = update_site<ALGO>(__ldcg(P + t.own1), __ldcg(P + t.offr1), __ldcg(P + t.own0),
                                             __ldcg(P + t.offu1), __ldcg(P + t.offd1), __ldcg(Pp + t.own1),
                                             __ldcg(Pm + t.own1) ^ fm, t.jr1, t.jr0, t.ju1, t.jd1, r.y, T);
        Sg[(size_t)p * L2 + t.own1] = v;
    }
}

}  // namespace

template <int ALGO>
__global__ void __launch_bounds__(512) k_sweep_wavefront(const Group g, const int C, const int nch, const int P,
                                                         const uint32_t sweep, const uint32_t k0, const uint32_t k1,
                                                         unsigned *__restrict__ arrivals) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ int do_boundary[32];
    const int L = g.L, L2 = L * L, Lt = g.Ltau, half = L / 2;
    const int tpu = L2 / 2;
    const int u = threadIdx.x / tpu, c = threadIdx.x - u * tpu;
    const int unit = blockIdx.x * P + u;
    const bool active = unit < g.nslots * nch;
    const int s = active ? unit / nch : 0;
    const int ch = active ? unit - s * nch : 0;
    const int a = ch * C, b = a + C;
    const int w = s / (g.R * g.K), j = s % g.K;
    uint64_t *ring = smem + (size_t)u * kRing * L2;
    uint64_t *Sg = g.S + (size_t)s * g.N;
    const Thr t = make_thr(g, c, w);
    uint32_t T[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) T[n] = g.thr[j * 16 + (ALGO == 0 ? n % 3 : 8 + n)];
    const uint32_t tag = (STREAM_SWEEP << 24) | ((uint32_t)g.gid << 8);
    const uint32_t qstride = (uint32_t)(L * half);
    const uint64_t apbc = g.boundary == 1 ? ~0ull : 0ull;

    auto slot_of = [&](int p) -> uint64_t * { return ring + ((p - a + 2) & (kRing - 1)) * L2; };
    auto issue = [&](int p) {
        if (active && p <= b) {
            const int gp = p < 0 ? p + Lt : (p >= Lt ? p - Lt : p);
            cp_async16(slot_of(p) + 2 * c, Sg + (size_t)gp * L2 + 2 * c);
        }
        cp_commit();
    };

    // prologue: planes a-1 .. a+kPrefetch-1
#pragma unroll
    for (int i = 0; i <= kPrefetch; ++i) issue(a - 1 + i);

    uint64_t W0[4], W1[4];  // own columns x0, x0+1 at planes tau-2 .. tau+1 (index = plane & 3)
    cp_wait<kPrefetch - 2>();
    __syncthreads();
    if (active) {
        W0[(a - 1) & 3] = slot_of(a - 1)[t.own0];
        W1[(a - 1) & 3] = slot_of(a - 1)[t.own1];
        W0[a & 3] = slot_of(a)[t.own0];
        W1[a & 3] = slot_of(a)[t.own1];
    }
    uint32_t o_y = 0, o_w = 0, carry = 0;

    // One step; I = tau & 3 is a compile-time constant in the unrolled loop.
#define QSG_WF_STEP(I)                                                                                            \
    {                                                                                                             \
        const int tau = base + (I);                                                                               \
        constexpr int IP1 = ((I) + 1) & 3, IM1 = ((I) + 3) & 3, IM2 = ((I) + 2) & 3;                             \
        cp_wait<kPrefetch - 2>();                                                                                 \
        __syncthreads();                                                                                          \
        if (active) {                                                                                             \
            const uint64_t *nxt = slot_of(tau + 1);                                                               \
            W0[IP1] = nxt[t.own0];                                                                                \
            W1[IP1] = nxt[t.own1];                                                                                \
        }                                                                                                         \
        issue(tau + kPrefetch);                                                                                   \
        if (active) {                                                                                             \
            uint64_t *pl = slot_of(tau);                                                                          \
            const uint64_t fp = tau == Lt - 1 ? apbc : 0ull, fm = tau == 0 ? apbc : 0ull;                         \
            if (((I) & 1) == 0) {                                                                                 \
                const uint4 r = philox4x32_10(make_uint4((uint32_t)(tau >> 1) * qstride + t.qrow, sweep,          \
                                                         (uint32_t)s, tag), k0, k1);                              \
                W0[I] = update_site<ALGO>(W0[I], W1[I], pl[t.offl0], pl[t.offu0], pl[t.offd0], W0[IP1] ^ fp,      \
                                          W0[IM1] ^ fm, t.jr0, t.jl0, t.ju0, t.jd0, r.x, T);                      \
                pl[t.own0] = W0[I];                                                                               \
                if (tau >= a + 2) {                                                                               \
                    uint64_t *pm = slot_of(tau - 1);                                                              \
                    W0[IM1] = update_site<ALGO>(W0[IM1], W1[IM1], pm[t.offl0], pm[t.offu0], pm[t.offd0], W0[I],   \
                                                W0[IM2], t.jr0, t.jl0, t.ju0, t.jd0, carry, T);                   \
                    pm[t.own0] = W0[IM1];                                                                         \
                }                                                                                                 \
                carry = r.z;                                                                                      \
                o_y = r.y;                                                                                        \
                o_w = r.w;                                                                                        \
            } else {                                                                                              \
                W1[I] = update_site<ALGO>(W1[I], pl[t.offr1], W0[I], pl[t.offu1], pl[t.offd1], W1[IP1] ^ fp,      \
                                          W1[IM1] ^ fm, t.jr1, t.jr0, t.ju1, t.jd1, o_w, T);                      \
                pl[t.own1] = W1[I];                                                                               \
                if (tau >= a + 2) {                                                                               \
                    uint64_t *pm = slot_of(tau - 1);                                                              \
                    W1[IM1] = update_site<ALGO>(W1[IM1], pm[t.offr1], W0[IM1], pm[t.offu1], pm[t.offd1], W1[I],   \
                                                W1[IM2], t.jr1, t.jr0, t.ju1, t.jd1, o_y, T);                     \
                    pm[t.own1] = W1[IM1];                                                                         \
                }                                                                                                 \
            }                                                                                                     \
            if (tau - 2 >= a) {                                                                                   \
                const uint64_t *wb = slot_of(tau - 2) + 2 * c;                                                    \
                *reinterpret_cast<ulonglong2 *>(Sg + (size_t)(tau - 2) * L2 + 2 * c) =                            \
                    *reinterpret_cast<const ulonglong2 *>(wb);                                                    \
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
            const uint64_t *wb = slot_of(p) + 2 * c;
            *reinterpret_cast<ulonglong2 *>(Sg + (size_t)p * L2 + 2 * c) = *reinterpret_cast<const ulonglong2 *>(wb);
        }
    }
    // arrival at the two chunk boundaries: the second unit to arrive updates them
    __threadfence();
    __syncthreads();
    if (c == 0) {
        int flags = 0;
        if (active) {
            const unsigned i0 = (unsigned)(s * nch + ch), i1 = (unsigned)(s * nch + (ch + 1 == nch ? 0 : ch + 1));
            if (atomicAdd(&arrivals[i0], 1u) == 1u) flags |= 1;
            if (atomicAdd(&arrivals[i1], 1u) == 1u) flags |= 2;
            __threadfence();
        }
        do_boundary[u] = flags;
    }
    __syncthreads();
    const int flags = do_boundary[u];
    if (active && flags) {
        if (flags & 1) boundary_update<ALGO>(g, t, Sg, a, T, sweep, (uint32_t)s, k0, k1);
        if (flags & 2) boundary_update<ALGO>(g, t, Sg, b == Lt ? 0 : b, T, sweep, (uint32_t)s, k0, k1);
        if (c == 0) {
            if (flags & 1) arrivals[s * nch + ch] = 0u;
            if (flags & 2) arrivals[s * nch + (ch + 1 == nch ? 0 : ch + 1)] = 0u;
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

size_t wavefront_smem_bytes(const Group &g, int P) { return (size_t)P * kRing * g.L * g.L * sizeof(uint64_t); }

int wavefront_units_per_block(const Group &g) {
    const int tpu = g.L * g.L / 2;
    int P = 1;
    while ((P * 2) * tpu <= 256 && P * 2 <= 16) P *= 2;
    return P;
}

cudaError_t launch_sweep_wavefront(const Group &g, uint32_t sweep, uint64_t seed, unsigned *arrivals, int C,
                                   cudaStream_t st) {
    const int nch = g.Ltau / C;
    const int P = wavefront_units_per_block(g);
    const int units = g.nslots * nch;
    const int blocks = (units + P - 1) / P;
    const size_t sm = wavefront_smem_bytes(g, P);
    const int threads = P * (g.L * g.L / 2);
    cudaError_t e;
    if (g.algo == 0) {
        e = cudaFuncSetAttribute(k_sweep_wavefront<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_sweep_wavefront<0><<<blocks, threads, sm, st>>>(g, C, nch, P, sweep, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                         arrivals);
    } else {
        e = cudaFuncSetAttribute(k_sweep_wavefront<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_sweep_wavefront<1><<<blocks, threads, sm, st>>>(g, C, nch, P, sweep, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                         arrivals);
    }
    return cudaGetLastError();
}

}  // namespace qsg
