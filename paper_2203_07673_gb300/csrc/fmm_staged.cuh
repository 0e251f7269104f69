// Staged row pass: the gathered rows of a team's next nonzeros wait in shared
// memory, copied there by cp.async, instead of in registers.
//
// The team kernel keeps U gathered rows per group in registers, so the rows
// in flight per SM are bounded by the register file; on patterns whose
// gathers mostly hit L2 (B about the L2 size) or whose rows are short, that
// bound (memory latency x rows in flight) sets the pass time, not HBM.  Here
// each lane copies its 16-byte vectors of the row of nonzero k + D - 1 into
// stage (k + D - 1) mod D of a ring in shared memory while nonzero k is used,
// so D gathers per team are in flight at a register cost of one row.  A lane
// only ever reads back the vectors it copied itself, so the per-thread
// cp.async.wait_group is the only synchronisation (no barrier, no wait that
// depends on another thread).  The column indices and values come in blocks
// of IB >= 16 consecutive nonzeros, one or two per lane, handed out by
// shuffles; the copies of nonzero k + D - 1 need the next block at most.
//
// Roles: FusedMM (the sampled dot product and the accumulation share the
// row), SDDMM and SpMM, over S or S^T, one team of G lanes per row or chunk
// (NG = 1).  Results are the same sums in the same order as the team kernel
// with one group per row.
#pragma once

#include <atomic>

#include "fmm_rows.cuh"

namespace fmm {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Widens this lane's VPL vectors of stage `st` (laid out [stage][v][thread]).
template <typename T, int VPL>
__device__ __forceinline__ void stage_read(const uint4 *ring, int st, int tid, float *f)
{
    constexpr int EPV = Elem<T>::PER16;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const uint4 q = ring[(st * VPL + v) * 256 + tid];
        if constexpr (sizeof(T) == 2) {
            unpack_bf16x8(q, f + v * EPV);
        } else {
            f[v * EPV + 0] = __uint_as_float(q.x); f[v * EPV + 1] = __uint_as_float(q.y);
            f[v * EPV + 2] = __uint_as_float(q.z); f[v * EPV + 3] = __uint_as_float(q.w);
        }
    }
}

template <int MODE, typename T, int R, int VPL, int D>
__global__ void __launch_bounds__(256) staged_pass_kernel(const PassArgs a)
{
    static_assert(MODE == M_FUSED || MODE == M_SDDMM || MODE == M_SPMM, "forward roles");
    using TS = TeamShape<T, R, VPL, 1>;
    constexpr int G = TS::G, E = TS::E, EPV = TS::EPV;
    constexpr int K = G >= 16 ? 1 : 16 / G;   // index entries per lane per block
    constexpr int IB = K * G;                 // nonzeros per index block
    static_assert(D >= 2 && D - 1 <= IB, "a copy D - 1 ahead needs at most the next block");
    constexpr bool HAS_L = MODE != M_SPMM;
    constexpr bool ACC = MODE != M_SDDMM;
    constexpr bool NZ = MODE == M_SDDMM;
    extern __shared__ uint4 ring[];   // [D][VPL][256]

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int lig = lane & (G - 1);
    const int tbase = lane & ~(G - 1);
    const long long gid = ((long long)blockIdx.x * blockDim.x + tid) / G;
    const long long total = (long long)a.n_chunks + a.n_light;
    const bool active = gid < total;
    const Loader ld;

    int row = 0, beg = 0, end = 0, slot = -1;
    if (active)
        pass_item(a, gid, row, beg, end, slot);
    const T *L = static_cast<const T *>(a.L);
    const T *Y = static_cast<const T *>(a.Y);
    float lrow[E], acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) { lrow[e] = 0.f; acc[e] = 0.f; }
    if (HAS_L && active && end > beg)
        team_load<T, VPL, G>(ld, L + (size_t)row * R, lig, lrow, false);

    const int n = end - beg;
    const int wn = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);

    // index block b: entry e of lane l is nonzero b * IB + e * G + l
    int jc[K], jn[K], ic[K], in_[K];
    float sc[K], sn[K];
    auto load_block = [&](int b, int (&j)[K], float (&s)[K], int (&si)[K]) {
#pragma unroll
        for (int e = 0; e < K; ++e) {
            const int q = b * IB + e * G + lig;
            j[e] = -1; s[e] = 0.f; si[e] = 0;
            if (q < n) {
                const int p = beg + q;
                j[e] = ld.idx(a.col_idx + p);
                // the slot in S order: for per-nonzero outputs, and for
                // values not yet in this CSR's order
                const int sp = (a.perm && (NZ || !a.s_direct)) ? ld.idx(a.perm + p) : p;
                si[e] = sp;
                s[e] = a.s ? ld.val(a.s + (a.s_direct ? p : sp)) : 1.f;
            }
        }
    };
    load_block(0, jc, sc, ic);
    load_block(1, jn, sn, in_);
    int cb = 0;   // index block of the nonzero being used

    // copies of nonzero k into stage k mod D (a commit group per nonzero,
    // empty past the end, so the group count stays uniform)
    auto issue = [&](int k) {
        const int o = k - cb * IB;   // < 2 IB
        const int e = (o < IB ? o : o - IB) / G;
        const int src = tbase + (o % G);
        const int jv = o < IB ? pick(jc, e) : pick(jn, e);
        const int j = __shfl_sync(0xffffffffu, jv, src);
        if (k < n && j >= 0) {
            const T *rowp = Y + (size_t)j * R;
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                cp_async16(&ring[((k % D) * VPL + v) * 256 + tid], rowp + (v * G + lig) * EPV);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < D - 1; ++k)
        issue(k);

    for (int k = 0; k < wn; ++k) {
        issue(k + D - 1);
        cp_async_wait<D - 1>();   // this thread's copies of nonzero k have landed
        const int o = k - cb * IB;
        const int e = o / G;
        const int src = tbase + (o % G);
        const int j = __shfl_sync(0xffffffffu, pick(jc, e), src);
        const float s = __shfl_sync(0xffffffffu, pick(sc, e), src);
        const int si = NZ ? __shfl_sync(0xffffffffu, pick(ic, e), src) : 0;
        const bool use = k < n && j >= 0;
        float y[E];
        if (use) {
            stage_read<T, VPL>(ring, k % D, tid, y);
        } else {
#pragma unroll
            for (int t = 0; t < E; ++t) y[t] = 0.f;
        }
        if constexpr (MODE == M_SPMM) {
            if (use) {
#pragma unroll
                for (int t = 0; t < E; ++t) acc[t] = fmaf(s, y[t], acc[t]);
            }
        } else {
            float d[1] = {0.f};
#pragma unroll
            for (int t = 0; t < E; ++t) d[0] = fmaf(lrow[t], y[t], d[0]);
            group_allreduce<G, 1>(d);
            if (use) {
                if constexpr (MODE == M_FUSED) {
                    const float c = s * d[0];
#pragma unroll
                    for (int t = 0; t < E; ++t) acc[t] = fmaf(c, y[t], acc[t]);
                } else {   // M_SDDMM
                    if (lig == (k % G))
                        nz_store<MODE>(a, si, s * d[0]);
                }
            }
        }
        if (o + 1 == IB) {
            // the next block becomes current; fetch the one after it
#pragma unroll
            for (int t = 0; t < K; ++t) { jc[t] = jn[t]; sc[t] = sn[t]; ic[t] = in_[t]; }
            ++cb;
            load_block(cb + 1, jn, sn, in_);
        }
    }
    cp_async_wait<0>();

    if constexpr (ACC) {
        if (active) {
            float *dst = slot >= 0 ? a.partials + (size_t)slot * R
                                   : (a.out ? a.out + (size_t)row * R : nullptr);
            if (dst)
                team_store_f32<T, VPL, G>(ld, dst, lig, acc, a.accumulate && slot < 0);
        }
    }
}

template <int MODE, typename T, int R, int VPL, int D>
cudaError_t launch_staged(const PassArgs &a, cudaStream_t st)
{
    constexpr int G = TeamShape<T, R, VPL, 1>::G;
    constexpr size_t smem = (size_t)D * VPL * 256 * 16;
    if constexpr (smem > 48 * 1024) {
        // more than the default dynamic shared memory: raise the kernel's
        // limit once per device (a bit per device of the first 64)
        static std::atomic<unsigned long long> done{0};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess)
            return e;
        const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
        if (!bit || !(done.load() & bit)) {
            e = cudaFuncSetAttribute(staged_pass_kernel<MODE, T, R, VPL, D>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return e;
            done.fetch_or(bit);
        }
    }
    const long long total = (long long)a.n_chunks + a.n_light;
    const long long blocks = (total * G + 255) / 256;
    staged_pass_kernel<MODE, T, R, VPL, D><<<(unsigned)blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int R>
cudaError_t dispatch_staged(int mode, int vpl, int stages, const PassArgs &a, cudaStream_t st)
{
    constexpr int B = base_vpl<T, R>();
#define FMM_STAGED(M, V, DD)                                                        \
    if constexpr (team_ok<T, R>(V, 1) && (DD - 1) <= 16)                            \
        if (mode == M && vpl == V && stages == DD)                                  \
            return launch_staged<M, T, R, V, DD>(a, st);
#define FMM_STAGED_MODES(V, DD) FMM_STAGED(M_FUSED, V, DD) FMM_STAGED(M_SDDMM, V, DD) FMM_STAGED(M_SPMM, V, DD)
    FMM_STAGED_MODES(B, 4) FMM_STAGED_MODES(B, 8) FMM_STAGED_MODES(2 * B, 4) FMM_STAGED_MODES(2 * B, 8)
#undef FMM_STAGED_MODES
#undef FMM_STAGED
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_staged_typed(int mode, int vpl_mult, int stages, const PassArgs &a,
                                cudaStream_t st)
{
    if ((long long)a.n_chunks + a.n_light == 0)
        return cudaSuccess;
    switch (a.r) {
    case 32: return dispatch_staged<T, 32>(mode, vpl_mult * base_vpl<T, 32>(), stages, a, st);
    case 64: return dispatch_staged<T, 64>(mode, vpl_mult * base_vpl<T, 64>(), stages, a, st);
    case 128: return dispatch_staged<T, 128>(mode, vpl_mult * base_vpl<T, 128>(), stages, a, st);
    case 256: return dispatch_staged<T, 256>(mode, vpl_mult * base_vpl<T, 256>(), stages, a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmm
