// Streaming row pass: a team walks a run of consecutive rows as one stream
// of nonzeros, with the register ring of the pipelined pass running across
// row boundaries.
//
// The row passes give each team one row: before its first multiply a team
// waits on a chain of loads (the row's place in the order, its row
// pointers, its column indices, then its gathered rows), and a row shorter
// than an index block still runs a whole block of batches.  On patterns of
// many short rows (Zipf-distributed rows, R-MAT graphs with half their rows
// empty) that per-row cost is a large part of the pass: the same nonzeros
// with groups of 4 to 8 consecutive rows merged into one run 25-38 % faster.
// Here the plan cuts the light rows (those not split into chunks) into runs
// of consecutive rows with at most kRunNnz nonzeros and kRunRows rows; a
// team takes one run and streams its nonzeros [row_ptr[first],
// row_ptr[end]) in index blocks of IB nonzeros, exactly as the pipelined
// pass streams one row's.  Before the nonzero at position p is used, the
// team finishes every row that ends at or before p: it stores that row's
// accumulator (zeros for an empty row), moves to the next row and takes the
// next row's local row, which it loaded one row ahead, as its own.  After
// the stream, the run's remaining rows are finished the same way.  Chunks of
// split rows are single-row streams whose accumulator goes to the partials.
//
// One nonzero per batch (a batch never straddles two rows), REFILL order of
// the ring, forward roles (FusedMM, SDDMM, SpMM).  The teams of a warp run
// the same number of batches (the longest stream of the warp; the plan
// orders runs by length so neighbours are alike); row changes are per team
// and touch only that team's registers and memory, so every shuffle is
// still reached by all lanes.
#pragma once

#include "fmm_pipe.cuh"

namespace fmm {

template <int MODE, typename T, int R, int VPL, int RING, int MB>
__global__ void __launch_bounds__(256, MB) stream_pass_kernel(const PassArgs a)
{
    static_assert(MODE == M_FUSED || MODE == M_SDDMM || MODE == M_SPMM, "forward roles");
    using TS = TeamShape<T, R, VPL, 1>;
    constexpr int G = TS::G, E = TS::E, EPV = TS::EPV;
    constexpr int E2 = E / 2, W2 = EPV / 2;   // float pairs per lane; per 16-byte word
    constexpr int K = G >= 8 ? 1 : 8 / G;     // index entries per lane per block
    constexpr int IB = K * G;                 // nonzeros per index block (one per batch)
    static_assert(IB % RING == 0, "ring layout");
    constexpr bool HAS_L = MODE != M_SPMM;
    constexpr bool ACC = MODE != M_SDDMM;
    constexpr bool NZ = MODE == M_SDDMM;
    constexpr bool WIDE = VPL % 2 == 0;       // lane-contiguous words, 32-byte loads

    const int lane = threadIdx.x & 31;
    const int lig = lane & (G - 1);
    const int tbase = lane & ~(G - 1);
    auto widx = [lig](int v) { return WIDE ? lig * VPL + v : v * G + lig; };
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long total = (long long)a.n_chunks + a.n_runs;
    const bool active = gid < total;
    const Loader ld;

    // the work item: rows [row, last) and their nonzeros [pbeg, pend)
    int row = 0, last = 0, pbeg = 0, pend = 0, slot = -1;
    int rend = 0, rend2 = 0;   // end of the current row's nonzeros, of the next row's
    if (active) {
        if (gid < a.n_chunks) {
            const int4 c = a.chunks[gid];
            row = c.x; last = c.x + 1; pbeg = c.y; pend = c.z; slot = (int)gid;
            rend = pend; rend2 = pend;
        } else {
            const int2 ru = a.runs[gid - a.n_chunks];
            row = ru.x; last = ru.y;
            pbeg = __ldg(a.row_ptr + row);
            pend = __ldg(a.row_ptr + last);
            rend = __ldg(a.row_ptr + row + 1);
            rend2 = __ldg(a.row_ptr + min(row + 2, last));
        }
    }
    int rbeg = pbeg;           // start of the current row's nonzeros
    const T *L = static_cast<const T *>(a.L);
    const T *Y = static_cast<const T *>(a.Y);

    float2 l2[E2], acc2[E2];
#pragma unroll
    for (int e = 0; e < E2; ++e) {
        l2[e] = make_float2(0.f, 0.f);
        acc2[e] = make_float2(0.f, 0.f);
    }
    // the next row's local row, loaded one row ahead (raw 16-byte words)
    uint4 lnext[HAS_L ? VPL : 1];
    auto load_local = [&](int rr, uint4 *w) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            w[v] = make_uint4(0u, 0u, 0u, 0u);
            if (rr < last)
                w[v] = ld.u4(reinterpret_cast<const uint4 *>(L + (size_t)rr * R) + widx(v), false);
        }
    };
    if constexpr (HAS_L) {
        if (active) {
            uint4 cur[VPL];
            load_local(row, cur);
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                unpack2<T>(cur[v], &l2[v * W2]);
            load_local(row + 1, lnext);
        } else {
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                lnext[v] = make_uint4(0u, 0u, 0u, 0u);
        }
    }

    // finish the current row (store its accumulator; an empty row stores
    // zeros, or nothing when accumulating) and move to the next
    auto finish_row = [&]() {
        if constexpr (ACC) {
            float *dst = slot >= 0 ? a.partials + (size_t)slot * R
                                   : (a.out ? a.out + (size_t)row * R : nullptr);
            const bool add = a.accumulate && slot < 0;
            if (dst && !(add && rend == rbeg)) {
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
#pragma unroll
                    for (int w = 0; w < W2; w += 2) {
                        const int k = widx(v) * EPV + 2 * w;
                        const float2 p0 = acc2[v * W2 + w], p1 = acc2[v * W2 + w + 1];
                        out_store4(ld, dst + k, make_float4(p0.x, p0.y, p1.x, p1.y), add);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E2; ++e)
                acc2[e] = make_float2(0.f, 0.f);
        }
        ++row;
        rbeg = rend;
        rend = rend2;
        if (slot < 0 && row + 1 < last)
            rend2 = __ldg(a.row_ptr + row + 2);
        if constexpr (HAS_L) {
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                unpack2<T>(lnext[v], &l2[v * W2]);
            load_local(row + 1, lnext);
        }
    };

    const int n = pend - pbeg;
    const int wn = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
    const int wblocks = (wn + IB - 1) / IB;

    // index block b of the stream: entry e of lane l is nonzero b * IB +
    // e * G + l; past the end j = -1 and s = 0
    int jc[K], jn[K], ic[K], in_[K];
    float sc[K], sn[K];
    float held[K];
#pragma unroll
    for (int e = 0; e < K; ++e) held[e] = 0.f;
    auto load_block = [&](int b, int (&j)[K], float (&s)[K], int (&si)[K]) {
#pragma unroll
        for (int e = 0; e < K; ++e) {
            const int q = b * IB + e * G + lig;
            j[e] = -1; s[e] = 0.f; si[e] = -1;
            if (q < n) {
                const int p = pbeg + q;
                j[e] = ld.idx(a.col_idx + p);
                const int sp = (a.perm && (NZ || !a.s_direct)) ? ld.idx(a.perm + p) : p;
                si[e] = sp;
                s[e] = a.s ? ld.val(a.s + (a.s_direct ? p : sp)) : 1.f;
            }
        }
    };

    uint4 ring[RING][VPL];
    // the gathered row of nonzero bb of the block whose indices are j
    auto issue = [&](uint4 (&dst)[VPL], const int (&j)[K], int bb) {
        const int jj = __shfl_sync(0xffffffffu, j[bb / G], tbase + (bb % G));
        if constexpr (WIDE) {
#pragma unroll
            for (int v = 0; v < VPL; v += 2) {
                dst[v] = make_uint4(0u, 0u, 0u, 0u);
                dst[v + 1] = make_uint4(0u, 0u, 0u, 0u);
                if (jj >= 0)
                    load32(reinterpret_cast<const uint4 *>(Y + (size_t)jj * R) + widx(v), dst[v],
                           dst[v + 1]);
            }
        } else {
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                dst[v] = make_uint4(0u, 0u, 0u, 0u);
                if (jj >= 0)
                    dst[v] = ld.u4(reinterpret_cast<const uint4 *>(Y + (size_t)jj * R) + widx(v), true);
            }
        }
    };

    load_block(0, jc, sc, ic);
    load_block(1, jn, sn, in_);
#pragma unroll
    for (int b = 0; b < RING; ++b)
        issue(ring[b], jc, b);

    for (int bk = 0; bk < wblocks; ++bk) {
#pragma unroll
        for (int bb = 0; bb < IB; ++bb) {
            const float sv = __shfl_sync(0xffffffffu, sc[bb / G], tbase + (bb % G));
            float2 y2[E2];
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                unpack2<T>(ring[bb % RING][v], &y2[v * W2]);
            // the slot just read takes the nonzero RING ahead (past this
            // block: from the next index block)
            {
                const int pf = bb + RING;
                if (pf < IB)
                    issue(ring[bb % RING], jc, pf);
                else
                    issue(ring[bb % RING], jn, pf - IB);
            }
            // rows that end before this nonzero are finished first
            const int q = bk * IB + bb;
            if (q < n) {
                while (pbeg + q >= rend && row + 1 < last)
                    finish_row();
            }
            if constexpr (MODE == M_SPMM) {
                const float2 c2 = make_float2(sv, sv);
#pragma unroll
                for (int e = 0; e < E2; ++e)
                    acc2[e] = ffma2(c2, y2[e], acc2[e]);
            } else {
                float2 t2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < E2; ++e)
                    t2 = ffma2(l2[e], y2[e], t2);
                float d = t2.x + t2.y;
#pragma unroll
                for (int off = G / 2; off > 0; off >>= 1)
                    d += __shfl_xor_sync(0xffffffffu, d, off);
                if constexpr (MODE == M_FUSED) {
                    const float c = sv * d;
                    const float2 c2 = make_float2(c, c);
#pragma unroll
                    for (int e = 0; e < E2; ++e)
                        acc2[e] = ffma2(c2, y2[e], acc2[e]);
                } else {   // M_SDDMM: the lane holding the nonzero's index entry keeps it
                    if (lig == bb % G)
                        held[bb / G] = sv * d;
                }
            }
        }
        if constexpr (NZ) {
#pragma unroll
            for (int e = 0; e < K; ++e)
                if (ic[e] >= 0)
                    nz_store<MODE>(a, ic[e], held[e]);
        }
        // the next block becomes current; fetch the one after it
#pragma unroll
        for (int e = 0; e < K; ++e) {
            jc[e] = jn[e]; sc[e] = sn[e]; ic[e] = in_[e];
        }
        load_block(bk + 2, jn, sn, in_);
    }
    // the rest of the run: the current row and any rows after it
    while (row < last)
        finish_row();
}

template <int MODE, typename T, int R, int VPL, int RING, int MB>
cudaError_t launch_stream(const PassArgs &a, cudaStream_t st)
{
    constexpr int G = TeamShape<T, R, VPL, 1>::G;
    const long long total = (long long)a.n_chunks + a.n_runs;
    const long long blocks = (total * G + 255) / 256;
    stream_pass_kernel<MODE, T, R, VPL, RING, MB><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Variants: (VPL as a multiple of the row shape's minimum, RING, MB).
template <typename T, int R>
cudaError_t dispatch_stream(int mode, int vpl, int ring, int mb, const PassArgs &a,
                            cudaStream_t st)
{
    constexpr int B = base_vpl<T, R>();
#define FMM_STREAM(M, V, RR, MM)                                                  \
    if constexpr (pipe_ok<T, R>(V, 1, RR))                                        \
        if (mode == M && vpl == V && ring == RR && mb == MM)                      \
            return launch_stream<M, T, R, V, RR, MM>(a, st);
#define FMM_STREAM_MODES(V, RR, MM)                                               \
    FMM_STREAM(M_FUSED, V, RR, MM) FMM_STREAM(M_SDDMM, V, RR, MM) FMM_STREAM(M_SPMM, V, RR, MM)
    FMM_STREAM_MODES(2 * B, 2, 2)
    FMM_STREAM_MODES(2 * B, 4, 2)
    FMM_STREAM_MODES(B, 2, 4)
#undef FMM_STREAM_MODES
#undef FMM_STREAM
    return cudaErrorNotSupported;   // not instantiated for this width: the caller falls back
}

template <typename T>
cudaError_t launch_stream_typed(int mode, int vpl_mult, int ring, int mb, const PassArgs &a,
                                cudaStream_t st)
{
    if ((long long)a.n_chunks + a.n_runs == 0)
        return cudaSuccess;
    switch (a.r) {
    case 32: return dispatch_stream<T, 32>(mode, vpl_mult * base_vpl<T, 32>(), ring, mb, a, st);
    case 64: return dispatch_stream<T, 64>(mode, vpl_mult * base_vpl<T, 64>(), ring, mb, a, st);
    case 128: return dispatch_stream<T, 128>(mode, vpl_mult * base_vpl<T, 128>(), ring, mb, a, st);
    case 256: return dispatch_stream<T, 256>(mode, vpl_mult * base_vpl<T, 256>(), ring, mb, a, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace fmm
