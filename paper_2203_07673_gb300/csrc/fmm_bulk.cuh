// Bulk-staged row pass: gathered rows are copied into shared memory by the
// bulk-copy engine (cp.async.bulk, one instruction per row) and wait there,
// not in registers.
//
// In the register-ring pass (fmm_pipe.cuh) every row in flight holds its
// lanes' registers, so rows in flight and teams per SM compete for one
// register file; on patterns whose gathers mostly hit L2 the pass is bound
// by that latency x concurrency product, not by bandwidth.  Here a team of G
// lanes owns a ring of D row slots in shared memory with one mbarrier per
// slot.  Lane 0 of the team starts the copy of the row of nonzero k + D into
// the slot that nonzero k has just released (mbarrier.arrive.expect_tx, then
// cp.async.bulk completing on that barrier); every lane waits for the slot's
// phase, reads its own 16-byte words with ld.shared and computes as the
// register-ring pass does (paired float32 FMAs).  A row costs one issue
// instruction per team and no registers while in flight.
//
// The grid is persistent (a multiple of the SM count): team t takes work
// items t, t + T, t + 2T, ... (T teams in the grid), all teams of a warp in
// lock step, so the shuffles see every lane.  The slots' barriers are set up
// once per team; each slot's phase parity is tracked in a bit mask.
//
// Every wait is bounded: after kWaitLimit unsuccessful polls the lane's warp
// stops starting copies and waiting (its remaining rows count as zeros) and
// records an error (*a.err = 1; fmm_plan_status reports it); before the
// block exits, lane 0 of each team waits again, bounded as well, for every
// copy it started and has not seen complete, so no copy lands in the shared
// memory of a block that has exited.
//
// No multicast, no cluster: every copy reads this GPU's memory into the
// issuing block's own shared memory.
//
// Roles: FusedMM, SDDMM, SpMM (the forward roles).
#pragma once

#include <atomic>

#include "fmm_pipe.cuh"

namespace fmm {

constexpr unsigned kWaitLimit = 1u << 22;   // polls of one slot before giving up

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(unsigned bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// Starts the copy of `bytes` bytes at src into the slot at dst, completing
// on the barrier bar (which expects exactly those bytes).
__device__ __forceinline__ void bulk_issue(unsigned dst, const void *src, unsigned bytes,
                                           unsigned bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Polls the barrier for the phase of the given parity, at most kWaitLimit
// times; true once the phase has completed.
__device__ __forceinline__ bool bar_wait(unsigned bar, unsigned parity)
{
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

template <int MODE, typename T, int R, int VPL, int D, int MB>
__global__ void __launch_bounds__(256, MB) bulk_pass_kernel(const PassArgs a)
{
    static_assert(MODE == M_FUSED || MODE == M_SDDMM || MODE == M_SPMM, "forward roles");
    using TS = TeamShape<T, R, VPL, 1>;
    constexpr int G = TS::G, E = TS::E, EPV = TS::EPV;
    constexpr int E2 = E / 2, W2 = EPV / 2;
    constexpr int ROW = R * (int)sizeof(T);   // bytes of one gathered row
    constexpr int TEAMS = 256 / G;            // teams per block
    constexpr int K = G >= 8 ? 1 : 8 / G;     // index entries per lane per block
    constexpr int IB = K * G;                 // nonzeros per index block
    static_assert(D >= 1 && D <= IB && (D & (D - 1)) == 0 && D <= 32, "ring depth");
    static_assert(ROW % 16 == 0, "bulk copies move multiples of 16 bytes");
    constexpr bool HAS_L = MODE != M_SPMM;
    constexpr bool ACC = MODE != M_SDDMM;
    constexpr bool NZ = MODE == M_SDDMM;

    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int lig = lane & (G - 1);
    const int tbase = lane & ~(G - 1);
    const int team = tid / G;
    const unsigned ring = smem_addr(smem + (size_t)team * D * ROW);
    const unsigned bars = smem_addr(smem + (size_t)TEAMS * D * ROW) + team * D * 8;
    const unsigned char *ring_g = smem + (size_t)team * D * ROW;

    if (lig == 0) {
#pragma unroll
        for (int d = 0; d < D; ++d)
            bar_init(bars + 8 * d);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    const long long teams_total = (long long)gridDim.x * TEAMS;
    const long long my_team = (long long)blockIdx.x * TEAMS + team;
    const long long total = (long long)a.n_chunks + a.n_light;
    const long long rounds = (total + teams_total - 1) / teams_total;
    const Loader ld;
    const T *L = static_cast<const T *>(a.L);
    const T *Y = static_cast<const T *>(a.Y);
    unsigned phases = 0;    // bit d: parity of the next phase of slot d
    unsigned pending = 0;   // bit d: a copy into slot d started and not seen complete
    bool failed = false;

    for (long long rd = 0; rd < rounds; ++rd) {
        const long long gid = my_team + rd * teams_total;
        const bool active = gid < total;
        int row = 0, beg = 0, end = 0, slot = -1;
        if (active)
            pass_item(a, gid, row, beg, end, slot);

        float2 l2[E2], acc2[E2];
#pragma unroll
        for (int e = 0; e < E2; ++e) {
            l2[e] = make_float2(0.f, 0.f);
            acc2[e] = make_float2(0.f, 0.f);
        }
        if (HAS_L && active && end > beg) {
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const uint4 q =
                    ld.u4(reinterpret_cast<const uint4 *>(L + (size_t)row * R) + v * G + lig, false);
                unpack2<T>(q, &l2[v * W2]);
            }
        }
        const int n = end - beg;
        const int wn = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);

        int jc[K], jn[K], ic[K], in_[K];
        float sc[K], sn[K];
        auto load_block = [&](int b, int (&j)[K], float (&s)[K], int (&si)[K]) {
#pragma unroll
            for (int e = 0; e < K; ++e) {
                const int q = b * IB + e * G + lig;
                j[e] = -1; s[e] = 0.f; si[e] = -1;
                if (q < n) {
                    const int p = beg + q;
                    j[e] = ld.idx(a.col_idx + p);
                    const int sp = (a.perm && (NZ || !a.s_direct)) ? ld.idx(a.perm + p) : p;
                    si[e] = sp;
                    s[e] = a.s ? ld.val(a.s + (a.s_direct ? p : sp)) : 1.f;
                }
            }
        };
        load_block(0, jc, sc, ic);
        load_block(1, jn, sn, in_);

        // the column of nonzero k (0 <= k - cb * IB < 2 IB) of this team
        auto column = [&](int k, int cb) {
            const int o = k - cb * IB;
            const int e = (o < IB ? o : o - IB) / G;
            const int src = tbase + (o % G);
            return __shfl_sync(0xffffffffu, o < IB ? pick(jc, e) : pick(jn, e), src);
        };
        // lane 0 starts the copy of the row of nonzero k into slot k % D
        auto start = [&](int k, int j) {
            if (lig == 0 && !failed && k < n && j >= 0) {
                const int d = k & (D - 1);
                bulk_issue(ring + d * ROW, Y + (size_t)j * R, ROW, bars + 8 * d);
                pending |= 1u << d;
            }
        };

        // the first D rows of the item (the ring is empty between items)
#pragma unroll
        for (int k = 0; k < D; ++k)
            start(k, column(k, 0));

        int cb = 0;
        for (int k = 0; k < wn; ++k) {
            const int o = k - cb * IB;
            const int e = o / G;
            const int src = tbase + (o % G);
            const float sv = __shfl_sync(0xffffffffu, pick(sc, e), src);
            const int sidx = NZ ? __shfl_sync(0xffffffffu, pick(ic, e), src) : -1;
            const int d = k & (D - 1);
            float2 y2[E2];
            bool use = k < n && !failed;
            bool ok = true;
            if (use) {
                ok = bar_wait(bars + 8 * d, (phases >> d) & 1u);
                if (ok) {
                    pending &= ~(1u << d);
                    phases ^= 1u << d;
                    const uint4 *w = reinterpret_cast<const uint4 *>(ring_g + d * ROW);
#pragma unroll
                    for (int v = 0; v < VPL; ++v)
                        unpack2<T>(w[v * G + lig], &y2[v * W2]);
                }
            }
            // a wait that gave up anywhere in the warp stops the warp's copies
            if (__any_sync(0xffffffffu, !ok))
                failed = true;
            use = use && ok;
            if (!use) {
#pragma unroll
                for (int t = 0; t < E2; ++t) y2[t] = make_float2(0.f, 0.f);
            }
            if constexpr (MODE == M_SPMM) {
                const float c = use ? sv : 0.f;
                const float2 c2 = make_float2(c, c);
#pragma unroll
                for (int t = 0; t < E2; ++t) acc2[t] = ffma2(c2, y2[t], acc2[t]);
            } else {
                float2 t2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < E2; ++t) t2 = ffma2(l2[t], y2[t], t2);
                float dd = t2.x + t2.y;
#pragma unroll
                for (int off = G / 2; off > 0; off >>= 1)
                    dd += __shfl_xor_sync(0xffffffffu, dd, off);
                if constexpr (MODE == M_FUSED) {
                    const float c = use ? sv * dd : 0.f;
                    const float2 c2 = make_float2(c, c);
#pragma unroll
                    for (int t = 0; t < E2; ++t) acc2[t] = ffma2(c2, y2[t], acc2[t]);
                } else {   // M_SDDMM
                    if (use && sidx >= 0 && lig == 0)
                        nz_store<MODE>(a, sidx, sv * dd);
                }
            }
            // every lane has read slot d (its values are in registers and
            // used above): it takes the row of nonzero k + D
            __syncwarp();
            start(k + D, column(k + D, cb));
            if (o + 1 == IB) {
#pragma unroll
                for (int t = 0; t < K; ++t) { jc[t] = jn[t]; sc[t] = sn[t]; ic[t] = in_[t]; }
                ++cb;
                load_block(cb + 1, jn, sn, in_);
            }
        }

        if constexpr (ACC) {
            if (active) {
                float *dst = slot >= 0 ? a.partials + (size_t)slot * R
                                       : (a.out ? a.out + (size_t)row * R : nullptr);
                if (dst) {
#pragma unroll
                    for (int v = 0; v < VPL; ++v) {
#pragma unroll
                        for (int w = 0; w < W2; w += 2) {
                            const int kk = (v * G + lig) * EPV + 2 * w;
                            const float2 p0 = acc2[v * W2 + w], p1 = acc2[v * W2 + w + 1];
                            out_store4(ld, dst + kk, make_float4(p0.x, p0.y, p1.x, p1.y),
                                       a.accumulate && slot < 0);
                        }
                    }
                }
            }
        }
    }

    // copies that a timed-out wait left behind: wait for them (bounded) so
    // none lands after the block has exited
    if (lig == 0 && pending) {
#pragma unroll 1
        for (int d = 0; d < D; ++d)
            if ((pending >> d) & 1u) {
                if (!bar_wait(bars + 8 * d, (phases >> d) & 1u))
                    failed = true;
            }
    }
    if (failed && a.err)
        atomicExch(a.err, 1);
}

template <int MODE, typename T, int R, int VPL, int D, int MB>
cudaError_t launch_bulk(const PassArgs &a, cudaStream_t st)
{
    constexpr int G = TeamShape<T, R, VPL, 1>::G;
    constexpr int TEAMS = 256 / G;
    constexpr size_t smem = (size_t)TEAMS * D * (R * sizeof(T)) + (size_t)TEAMS * D * 8;
    if constexpr (smem > 48 * 1024) {
        static std::atomic<unsigned long long> done{0};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess)
            return e;
        const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
        if (!bit || !(done.load() & bit)) {
            e = cudaFuncSetAttribute(bulk_pass_kernel<MODE, T, R, VPL, D, MB>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return e;
            done.fetch_or(bit);
        }
    }
    const long long total = (long long)a.n_chunks + a.n_light;
    const long long need = (total + TEAMS - 1) / TEAMS;
    const long long grid = std::min<long long>(need, (long long)sm_count() * MB);
    bulk_pass_kernel<MODE, T, R, VPL, D, MB><<<(unsigned)std::max<long long>(grid, 1), 256, smem, st>>>(a);
    return cudaGetLastError();
}

// Whether (VPL, D, MB) fits rows of R elements of T: a valid team layout,
// a ring no deeper than the index block, and MB blocks' shared memory
// within the 227 KB an SM offers.
template <typename T, int R>
constexpr bool bulk_ok(int V, int D, int MB)
{
    if (!team_ok<T, R>(V, 1))
        return false;
    const int g = R * (int)sizeof(T) / 16 / V;
    const int ib = g >= 8 ? g : 8;
    const long long smem = (long long)(256 / g) * D * (R * (long long)sizeof(T) + 8);
    return D <= ib && smem * MB <= 227 * 1024;
}

// Variants: (VPL, D, MB) with VPL as a multiple of the row shape's minimum.
template <typename T, int R>
cudaError_t dispatch_bulk(int mode, int vpl, int depth, int mb, const PassArgs &a, cudaStream_t st)
{
    constexpr int B = base_vpl<T, R>();
#define FMM_BULK(M, V, DD, MM)                                                      \
    if constexpr (bulk_ok<T, R>(V, DD, MM))                                         \
        if (mode == M && vpl == V && depth == DD && mb == MM)                       \
            return launch_bulk<M, T, R, V, DD, MM>(a, st);
#define FMM_BULK_MODES(V, DD, MM) \
    FMM_BULK(M_FUSED, V, DD, MM) FMM_BULK(M_SDDMM, V, DD, MM) FMM_BULK(M_SPMM, V, DD, MM)
    FMM_BULK_MODES(2 * B, 4, 4)
    FMM_BULK_MODES(2 * B, 8, 3)
    FMM_BULK_MODES(B, 4, 4)
    FMM_BULK_MODES(B, 8, 4)
#undef FMM_BULK_MODES
#undef FMM_BULK
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_bulk_typed(int mode, int vpl_mult, int depth, int mb, const PassArgs &a,
                              cudaStream_t st)
{
    if ((long long)a.n_chunks + a.n_light == 0)
        return cudaSuccess;
    switch (a.r) {
    case 32: return dispatch_bulk<T, 32>(mode, vpl_mult * base_vpl<T, 32>(), depth, mb, a, st);
    case 64: return dispatch_bulk<T, 64>(mode, vpl_mult * base_vpl<T, 64>(), depth, mb, a, st);
    case 128: return dispatch_bulk<T, 128>(mode, vpl_mult * base_vpl<T, 128>(), depth, mb, a, st);
    case 256: return dispatch_bulk<T, 256>(mode, vpl_mult * base_vpl<T, 256>(), depth, mb, a, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace fmm
