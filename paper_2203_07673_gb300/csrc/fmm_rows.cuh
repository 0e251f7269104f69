// Row-pass kernels of libfmm.
//
// Every operation of the library is one "row pass" over a CSR (S, or S^T with
// a permutation back to the CSR slots of S): a group of G lanes owns one
// output row (or one chunk of a split row), keeps that row's local operands
// in registers, and walks the row's nonzeros U at a time.  For each nonzero
// it gathers one dense row through col_idx with 16-byte loads, forms the
// sampled inner products with per-lane partial sums and an xor-shuffle
// reduction inside the group, and folds the result into a register
// accumulator.  The output row is written once.  This is the local kernel
// fusion of Sec. IV-B (2): in the fused roles the SDDMM value of a nonzero
// (Sec. II, Eq. 1) lives in a register for the few instructions between the
// reduction and the accumulation, and never reaches memory.
//
// Roles (Mode):
//   M_FUSED    acc += s * <L_i, Y_j> * Y_j          FusedMMA / FusedMMB
//   M_SDDMM    v[p] = s * <L_i, Y_j>                SDDMM (Eq. 1)
//   M_SPMM     acc += v[p] * Y_j                    SpMMA / SpMMB
//   M_BWD_ROW  ds[p] = <L_i,Y_j> <H_i,Y_j>;  acc += s <H_i,Y_j> Y_j
//   M_BWD_COL  acc += s (<Y_i,L_j> H_i + <H_i,L_j> Y_i)   (H_i gathered too)
#pragma once

#include "fmm_internal.cuh"

namespace fmm {

typedef uint16_t bf16_t;   // bfloat16 bits

template <typename T> struct Elem;
template <> struct Elem<float> { static constexpr int PER16 = 4; };
template <> struct Elem<bf16_t> { static constexpr int PER16 = 8; };

// Lane layout of one dense row of r elements of type T: the row is split
// into 16-byte vectors; a group of G lanes (G = min(32, vectors)) owns it,
// lane l holding vectors l, l + G, ...  Element k of lane l, vector v,
// position t is k = (v * G + l) * EPV + t.
template <typename T, int R>
struct Shape {
    static constexpr int ROW_BYTES = R * (int)sizeof(T);
    static constexpr int VECS = ROW_BYTES / 16;
    static constexpr int G = VECS < 32 ? VECS : 32;
    static constexpr int VPL = VECS / G;
    static constexpr int EPV = Elem<T>::PER16;
    static constexpr int E = VPL * EPV;
    static_assert(ROW_BYTES % 16 == 0 && VECS % G == 0, "unsupported r");
};

__device__ __forceinline__ void unpack_bf16x8(const uint4 q, float *f)
{
    f[0] = __uint_as_float(q.x << 16); f[1] = __uint_as_float(q.x & 0xffff0000u);
    f[2] = __uint_as_float(q.y << 16); f[3] = __uint_as_float(q.y & 0xffff0000u);
    f[4] = __uint_as_float(q.z << 16); f[5] = __uint_as_float(q.z & 0xffff0000u);
    f[6] = __uint_as_float(q.w << 16); f[7] = __uint_as_float(q.w & 0xffff0000u);
}

// Row loads and stores with fixed cache operators: STREAM = read once
// (ld.global.cs), else the read-only path.
template <typename T, int R, bool STREAM>
__device__ __forceinline__ void load_row(const T *row, int lig, float (&f)[Shape<T, R>::E])
{
    using S = Shape<T, R>;
#pragma unroll
    for (int v = 0; v < S::VPL; ++v) {
        const int vec = v * S::G + lig;
        if constexpr (sizeof(T) == 4) {
            const float4 *p = reinterpret_cast<const float4 *>(row) + vec;
            const float4 q = STREAM ? __ldcs(p) : __ldg(p);
            f[v * 4 + 0] = q.x; f[v * 4 + 1] = q.y; f[v * 4 + 2] = q.z; f[v * 4 + 3] = q.w;
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(row) + vec;
            const uint4 q = STREAM ? __ldcs(p) : __ldg(p);
            unpack_bf16x8(q, &f[v * 8]);
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void store_row_f32(float *row, int lig, const float (&f)[Shape<T, R>::E])
{
    using S = Shape<T, R>;
#pragma unroll
    for (int v = 0; v < S::VPL; ++v) {
#pragma unroll
        for (int q = 0; q < S::EPV / 4; ++q) {
            const int k = (v * S::G + lig) * S::EPV + 4 * q;
            const int e = v * S::EPV + 4 * q;
            __stcs(reinterpret_cast<float4 *>(row + k),
                   make_float4(f[e + 0], f[e + 1], f[e + 2], f[e + 3]));
        }
    }
}

// Sum over the G lanes of a group (xor butterfly; every lane gets the sum).
template <int G, int NV>
__device__ __forceinline__ void group_allreduce(float (&v)[NV])
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < NV; ++i)
            v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    }
}

// Element e of a small register array (a select chain, so the array stays
// in registers when e is not a compile-time constant).
template <int K>
__device__ __forceinline__ int pick(const int (&x)[K], int e)
{
    int r = x[0];
#pragma unroll
    for (int i = 1; i < K; ++i)
        if (e == i) r = x[i];
    return r;
}
template <int K>
__device__ __forceinline__ float pick(const float (&x)[K], int e)
{
    float r = x[0];
#pragma unroll
    for (int i = 1; i < K; ++i)
        if (e == i) r = x[i];
    return r;
}

// A per-nonzero output: SDDMM values are added to what v holds in the
// accumulating calls (the partial dot products of the sparse-shifting
// algorithm); ds is always overwritten.
template <int MODE>
__device__ __forceinline__ void nz_store(const PassArgs &a, int slot, float v)
{
    if (MODE == M_SDDMM && a.accumulate)
        a.nzout[slot] += v;
    else
        a.nzout[slot] = v;
}

// Work item of group `gid`: chunks of split rows first, then light rows in
// plan order.  slot >= 0 marks a chunk (its partial row goes to partials).
__device__ __forceinline__ void pass_item(const PassArgs &a, long long gid, int &row,
                                          int &beg, int &end, int &slot)
{
    if (gid < a.n_chunks) {
        const int4 c = a.chunks[gid];
        row = c.x; beg = c.y; end = c.z; slot = (int)gid;
    } else {
        row = a.order[gid - a.n_chunks];
        beg = __ldg(a.row_ptr + row);
        end = __ldg(a.row_ptr + row + 1);
        slot = -1;
    }
}

// Cache operators of the row passes: gathered rows and CSR arrays take the
// read-only path (ld.global.nc); local rows, read once, and outputs, written
// once, are evict-first (ld/st.global.cs).
struct Loader {
    __device__ __forceinline__ int idx(const int32_t *p) const { return __ldg(p); }
    __device__ __forceinline__ float val(const float *p) const { return __ldg(p); }
    __device__ __forceinline__ float4 f4(const void *p, bool gather) const
    {
        const float4 *q = static_cast<const float4 *>(p);
        return gather ? __ldg(q) : __ldcs(q);
    }
    __device__ __forceinline__ uint4 u4(const void *p, bool gather) const
    {
        const uint4 *q = static_cast<const uint4 *>(p);
        return gather ? __ldg(q) : __ldcs(q);
    }
    __device__ __forceinline__ void st4(float *p, float4 v) const
    {
        __stcs(reinterpret_cast<float4 *>(p), v);
    }
};

// Team layout of one dense row of R elements of type T: VECS 16-byte vectors
// held by a group of G = VECS / VPL lanes, lane l owning vectors l, l + G, ...
// (element k = (v * G + l) * EPV + t).  A team of NG groups owns one output
// row; group g takes nonzeros g, g + NG, ... of that row.
template <typename T, int R, int VPL, int NG>
struct TeamShape {
    static constexpr int VECS = R * (int)sizeof(T) / 16;
    static constexpr int G = VECS / VPL;
    static constexpr int TEAM = G * NG;
    static constexpr int EPV = Elem<T>::PER16;
    static constexpr int E = VPL * EPV;
    static_assert(R * (int)sizeof(T) % 16 == 0 && VECS % VPL == 0 && G >= 1, "layout");
    static_assert(TEAM <= 32 && 32 % TEAM == 0 && (G & (G - 1)) == 0, "team");
};

template <typename T, int VPL, int G>
__device__ __forceinline__ void team_load(const Loader &ld, const T *row, int lig, float *f,
                                          bool gather)
{
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int vec = v * G + lig;
        if constexpr (sizeof(T) == 4) {
            const float4 q = ld.f4(reinterpret_cast<const float4 *>(row) + vec, gather);
            f[v * 4 + 0] = q.x; f[v * 4 + 1] = q.y; f[v * 4 + 2] = q.z; f[v * 4 + 3] = q.w;
        } else {
            const uint4 q = ld.u4(reinterpret_cast<const uint4 *>(row) + vec, gather);
            unpack_bf16x8(q, &f[v * 8]);
        }
    }
}

// A float32 row (gradients, outputs) with the element mapping of T.
template <typename T, int VPL, int G>
__device__ __forceinline__ void team_load_f32(const Loader &ld, const float *row, int lig,
                                              float *f, bool gather)
{
    constexpr int EPV = Elem<T>::PER16;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
#pragma unroll
        for (int q = 0; q < EPV / 4; ++q) {
            const float4 x = ld.f4(row + (v * G + lig) * EPV + 4 * q, gather);
            f[v * EPV + 4 * q + 0] = x.x; f[v * EPV + 4 * q + 1] = x.y;
            f[v * EPV + 4 * q + 2] = x.z; f[v * EPV + 4 * q + 3] = x.w;
        }
    }
}

// Stores four output elements; with add, adds them to what the row holds
// (the accumulating calls: out += the pass).
__device__ __forceinline__ void out_store4(const Loader &ld, float *p, float4 v, bool add)
{
    if (add) {
        const float4 o = __ldcs(reinterpret_cast<const float4 *>(p));
        v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
    }
    ld.st4(p, v);
}

template <typename T, int VPL, int G>
__device__ __forceinline__ void team_store_f32(const Loader &ld, float *row, int lig,
                                               const float *f, bool add = false)
{
    constexpr int EPV = Elem<T>::PER16;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
#pragma unroll
        for (int q = 0; q < EPV / 4; ++q) {
            const int e = v * EPV + 4 * q;
            out_store4(ld, row + (v * G + lig) * EPV + 4 * q,
                       make_float4(f[e + 0], f[e + 1], f[e + 2], f[e + 3]), add);
        }
    }
}

// One row pass.  A team of NG x G lanes owns one work item (a light row, or
// a chunk of a split row); per batch each group handles U nonzeros, so a
// batch covers NG * U consecutive nonzeros (nonzero base + u * NG + g goes to
// group g).  Gathers of a batch are all issued before any is used.  After the
// last batch the NG partial accumulators are summed across the team and
// group 0 stores the row.
//
// team_pass_body does the work of team `gid` (every lane of the warp must
// call it; lanes whose team is not active only join the shuffles).
template <int MODE, typename T, int R, int VPL, int NG, int U>
__device__ __forceinline__ void team_pass_body(const PassArgs &a, long long gid, bool active)
{
    using TS = TeamShape<T, R, VPL, NG>;
    constexpr int G = TS::G, TEAM = TS::TEAM, E = TS::E;
    constexpr bool HAS_L = MODE != M_SPMM;
    constexpr bool ACC = MODE != M_SDDMM;
    constexpr bool TWO = MODE == M_BWD_ROW || MODE == M_BWD_COL;
    constexpr int ND = TWO ? 2 * U : U;
    (void)TEAM;

    const int lane = threadIdx.x & 31;
    const int lig = lane & (G - 1);
    const int grp = (lane / G) & (NG - 1);
    const Loader ld;

    int row = 0, beg = 0, end = 0, slot = -1;
    if (active)
        pass_item(a, gid, row, beg, end, slot);

    const T *L = static_cast<const T *>(a.L);
    const T *Y = static_cast<const T *>(a.Y);

    float lrow[E], hrow[TWO ? E : 1], acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) { lrow[e] = 0.f; acc[e] = 0.f; }
#pragma unroll
    for (int e = 0; e < (TWO ? E : 1); ++e) hrow[e] = 0.f;
    // rows without nonzeros only write zeros: their local rows are not read
    if (HAS_L && active && end > beg)
        team_load<T, VPL, G>(ld, L + (size_t)row * R, lig, lrow, false);
    if constexpr (MODE == M_BWD_ROW)
        if (active && end > beg)
            team_load_f32<T, VPL, G>(ld, a.H + (size_t)row * R, lig, hrow, false);

    constexpr int PER = NG * U;
    constexpr bool NZ = MODE == M_SDDMM || MODE == M_BWD_ROW;
    // Per-nonzero outputs (v, ds).  With one group per team and the team's
    // index blocks, the lane that loaded a nonzero's index keeps its value
    // (owner == the nonzero's position in the block) and the team stores a
    // block of values at once (HOLD); otherwise each value is stored as it
    // is computed.
    constexpr bool HOLD = NZ && NG == 1 && TEAM % PER == 0;
    float held = 0.f;
    // one batch: the gathers of its U nonzeros per group, then their use;
    // `first` is the position in the team's index block of its nonzero 0
    auto batch = [&](const int (&jj)[U], const int (&sidx)[U], const float (&sv)[U], int first) {
        float y[U][E];
        float h[MODE == M_BWD_COL ? U : 1][E];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= 0) {
                team_load<T, VPL, G>(ld, Y + (size_t)jj[u] * R, lig, y[u], true);
                if constexpr (MODE == M_BWD_COL)
                    team_load_f32<T, VPL, G>(ld, a.H + (size_t)jj[u] * R, lig, h[u], true);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    y[u][e] = 0.f;
                    if constexpr (MODE == M_BWD_COL) h[u][e] = 0.f;
                }
            }
        }
        if constexpr (MODE == M_SPMM) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (jj[u] >= 0) {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        acc[e] = fmaf(sv[u], y[u][e], acc[e]);
                }
        } else {
            float d[ND];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float t = 0.f;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    t = fmaf(lrow[e], y[u][e], t);
                d[u] = t;
                if constexpr (MODE == M_BWD_ROW) {
                    float w = 0.f;
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        w = fmaf(hrow[e], y[u][e], w);
                    d[U + u] = w;
                } else if constexpr (MODE == M_BWD_COL) {
                    float w = 0.f;
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        w = fmaf(h[u][e], lrow[e], w);
                    d[U + u] = w;
                }
            }
            group_allreduce<G, ND>(d);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jj[u] < 0)
                    continue;
                if constexpr (MODE == M_FUSED) {
                    const float c = sv[u] * d[u];
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        acc[e] = fmaf(c, y[u][e], acc[e]);
                } else if constexpr (MODE == M_SDDMM) {
                    if constexpr (HOLD) {
                        if ((lane & (TEAM - 1)) == first + u)
                            held = sv[u] * d[u];
                    } else if (lig == (u % G)) {
                        nz_store<MODE>(a, sidx[u], sv[u] * d[u]);
                    }
                } else if constexpr (MODE == M_BWD_ROW) {
                    if constexpr (HOLD) {
                        if ((lane & (TEAM - 1)) == first + u)
                            held = d[u] * d[U + u];
                    } else if (a.nzout && lig == (u % G)) {
                        a.nzout[sidx[u]] = d[u] * d[U + u];
                    }
                    const float c = sv[u] * d[U + u];
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        acc[e] = fmaf(c, y[u][e], acc[e]);
                } else {  // M_BWD_COL
                    const float c1 = sv[u] * d[u], c2 = sv[u] * d[U + u];
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        acc[e] = fmaf(c1, h[u][e], fmaf(c2, y[u][e], acc[e]));
                }
            }
        }
    };

    if constexpr (TEAM % PER == 0) {
        // The team loads the column indices (and values, and S-order slots)
        // of TEAM consecutive nonzeros at once, one per lane, coalesced, and
        // hands them to its groups by shuffles: the index latency is paid
        // once per TEAM / PER batches instead of once per batch.
        constexpr int SUB = TEAM / PER;
        const int tl = lane & (TEAM - 1);
        const int tbase = lane & ~(TEAM - 1);
        const int blocks = (end - beg + TEAM - 1) / TEAM;
        const int wblocks = (int)__reduce_max_sync(0xffffffffu, (unsigned)blocks);
        for (int bk = 0; bk < wblocks; ++bk) {
            const int q = beg + bk * TEAM + tl;
            int myj = -1, mysi = 0;
            float mys = 0.f;
            if (q < end) {
                myj = ld.idx(a.col_idx + q);
                // the slot in S order is needed for per-nonzero outputs and
                // for values not yet in this CSR's order
                mysi = (a.perm && (NZ || !a.s_direct)) ? ld.idx(a.perm + q) : q;
                mys = a.s ? ld.val(a.s + (a.s_direct ? q : mysi)) : 1.f;
            }
#pragma unroll 1
            for (int sub = 0; sub < SUB; ++sub) {
                int jj[U], sidx[U];
                float sv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int src = tbase + sub * PER + u * NG + grp;
                    jj[u] = __shfl_sync(0xffffffffu, myj, src);
                    sv[u] = __shfl_sync(0xffffffffu, mys, src);
                    sidx[u] = (NZ && !HOLD) ? __shfl_sync(0xffffffffu, mysi, src) : 0;
                }
                batch(jj, sidx, sv, sub * PER);
            }
            // the block's per-nonzero outputs, one store per lane
            if constexpr (HOLD)
                if (q < end && a.nzout)
                    nz_store<MODE>(a, mysi, held);
        }
    } else {
        const int iters = (end - beg + PER - 1) / PER;
        const int witers = (int)__reduce_max_sync(0xffffffffu, (unsigned)iters);
        for (int it = 0; it < witers; ++it) {
            const int p0 = beg + it * PER + grp;
            int jj[U], sidx[U];
            float sv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = p0 + u * NG;
                if (p < end) {
                    jj[u] = ld.idx(a.col_idx + p);
                    sidx[u] = (a.perm && (NZ || !a.s_direct)) ? ld.idx(a.perm + p) : p;
                    sv[u] = a.s ? ld.val(a.s + (a.s_direct ? p : sidx[u])) : 1.f;
                } else {
                    jj[u] = -1; sidx[u] = 0; sv[u] = 0.f;
                }
            }
            batch(jj, sidx, sv, 0);
        }
    }

    if constexpr (ACC) {
        // partial rows of the NG groups, summed in a fixed xor order
#pragma unroll
        for (int off = G; off < TEAM; off <<= 1) {
#pragma unroll
            for (int e = 0; e < E; ++e)
                acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
        }
        if (active && grp == 0) {
            float *dst = slot >= 0 ? a.partials + (size_t)slot * R
                                   : (a.out ? a.out + (size_t)row * R : nullptr);
            if (dst)
                team_store_f32<T, VPL, G>(ld, dst, lig, acc, a.accumulate && slot < 0);
        }
    }
}

// Blocks of 256 threads that a row pass asks to keep resident per SM (a
// register cap of 65536 / (256 x blocks) per thread).  Only light variants
// (at most 40 floats live per lane) are capped: forward-type passes at 5
// blocks (48 registers), the backward pass over S at 4 (64); the backward
// pass over S^T, with two gathered rows per nonzero, spills when capped.
// Measured on GB300 against the uncapped build: FusedMMA 14 % faster on
// Zipf rows, 10 % on R-MAT and 2 % on Erdos-Renyi rows; the backward pass
// over S 9-16 % faster.
template <int MODE, typename T, int R, int VPL, int NG, int U>
constexpr int team_min_blocks()
{
    constexpr int E = VPL * Elem<T>::PER16;
    constexpr int live = E * (U * (MODE == M_BWD_COL ? 2 : 1) + 2 + (MODE == M_BWD_ROW ? 1 : 0));
    if (live > 40)
        return 1;
    return MODE == M_BWD_COL ? 1 : MODE == M_BWD_ROW ? 4 : 5;
}

// Blocks of two warps: small blocks retire as soon as their rows are done,
// so the SM starts new rows sooner (GB300, against 256-thread blocks: Zipf
// rows FP32 FusedMMA 1.677 -> 1.645 ms, R-MAT backward 5.13 -> 5.00 ms with
// the register-ring pass).  The register caps of team_min_blocks keep their
// meaning: 256 / kTeamBlock blocks per 256 threads.
constexpr int kTeamBlock = 64;

template <int MODE, typename T, int R, int VPL, int NG, int U>
__global__ void __launch_bounds__(kTeamBlock,
                                  (256 / kTeamBlock) * (team_min_blocks<MODE, T, R, VPL, NG, U>()))
    team_pass_kernel(const PassArgs a)
{
    constexpr int TEAM = TeamShape<T, R, VPL, NG>::TEAM;
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TEAM;
    const long long total = (long long)a.n_chunks + a.n_light;
    team_pass_body<MODE, T, R, VPL, NG, U>(a, gid, gid < total);
}

template <typename T> __device__ __forceinline__ float widen(T x);
template <> __device__ __forceinline__ float widen<float>(float x) { return x; }
template <> __device__ __forceinline__ float widen<bf16_t>(bf16_t x)
{
    return __uint_as_float(((uint32_t)x) << 16);
}

__device__ __forceinline__ float warp_allreduce(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Generic pass for any r and any alignment: one warp per row or chunk,
// scalar loads strided by lane, the output row accumulated in place (each
// lane owns the columns k = lane + 32 t, so no two lanes touch one word).
template <int MODE, typename T>
__global__ void __launch_bounds__(256) row_pass_generic(const PassArgs a)
{
    constexpr bool ACC = MODE != M_SDDMM;
    const int lane = threadIdx.x & 31;
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long total = (long long)a.n_chunks + a.n_light;
    if (gid >= total)
        return;   // uniform per warp
    int row, beg, end, slot;
    pass_item(a, gid, row, beg, end, slot);
    const int r = a.r;
    const T *L = static_cast<const T *>(a.L);
    const T *Y = static_cast<const T *>(a.Y);
    float *dst = nullptr;
    if (ACC)
        dst = slot >= 0 ? a.partials + (size_t)slot * r
                        : (a.out ? a.out + (size_t)row * r : nullptr);
    // the accumulating calls add into the output row as it stands
    if (dst && !(a.accumulate && slot < 0))
        for (int k = lane; k < r; k += 32)
            dst[k] = 0.f;
    const T *Li = L ? L + (size_t)row * r : nullptr;
    for (int p = beg; p < end; ++p) {
        const int j = __ldg(a.col_idx + p);
        const int sidx = a.perm ? __ldg(a.perm + p) : p;
        const float sv = a.s ? __ldg(a.s + (a.s_direct ? p : sidx)) : 1.f;
        const T *Yj = Y + (size_t)j * r;
        float d = 0.f, w = 0.f;
        if constexpr (MODE != M_SPMM) {
            for (int k = lane; k < r; k += 32) {
                const float yk = widen<T>(Yj[k]);
                d = fmaf(widen<T>(Li[k]), yk, d);
                if constexpr (MODE == M_BWD_ROW)
                    w = fmaf(a.H[(size_t)row * r + k], yk, w);
                if constexpr (MODE == M_BWD_COL)
                    w = fmaf(a.H[(size_t)j * r + k], widen<T>(Li[k]), w);
            }
            d = warp_allreduce(d);
            if constexpr (MODE == M_BWD_ROW || MODE == M_BWD_COL)
                w = warp_allreduce(w);
        }
        if constexpr (MODE == M_SDDMM) {
            if (lane == 0)
                nz_store<MODE>(a, sidx, sv * d);
        } else if constexpr (MODE == M_BWD_ROW) {
            if (lane == 0 && a.nzout)
                a.nzout[sidx] = d * w;
        }
        if (dst) {
            if constexpr (MODE == M_FUSED) {
                const float c = sv * d;
                for (int k = lane; k < r; k += 32)
                    dst[k] = fmaf(c, widen<T>(Yj[k]), dst[k]);
            } else if constexpr (MODE == M_SPMM) {
                for (int k = lane; k < r; k += 32)
                    dst[k] = fmaf(sv, widen<T>(Yj[k]), dst[k]);
            } else if constexpr (MODE == M_BWD_ROW) {
                const float c = sv * w;
                for (int k = lane; k < r; k += 32)
                    dst[k] = fmaf(c, widen<T>(Yj[k]), dst[k]);
            } else if constexpr (MODE == M_BWD_COL) {
                const float c1 = sv * d, c2 = sv * w;
                for (int k = lane; k < r; k += 32)
                    dst[k] = fmaf(c1, a.H[(size_t)j * r + k],
                                  fmaf(c2, widen<T>(Yj[k]), dst[k]));
            }
        }
    }
}

// Kernel variants of the vectorised path: (VPL, NG, U) = vectors per lane,
// groups per team, nonzeros per group per batch.  Variant 0 picks the
// default of the row shape; the others are listed in kVariants.
struct Variant {
    int vpl, ng, u;
};

template <int MODE, typename T, int R, int VPL, int NG, int U>
cudaError_t launch_team(const PassArgs &a, cudaStream_t st)
{
    constexpr int TEAM = TeamShape<T, R, VPL, NG>::TEAM;
    const long long total = (long long)a.n_chunks + a.n_light;
    const long long blocks = (total * TEAM + kTeamBlock - 1) / kTeamBlock;
    team_pass_kernel<MODE, T, R, VPL, NG, U><<<(unsigned)blocks, kTeamBlock, 0, st>>>(a);
    return cudaGetLastError();
}

// Whether (VPL, NG) is a valid team layout for rows of R elements of T.
template <typename T, int R>
constexpr bool team_ok(int V, int N)
{
    const int vecs = R * (int)sizeof(T) / 16;
    if (V < 1 || vecs % V != 0) return false;
    const int g = vecs / V;
    return g >= 1 && (g & (g - 1)) == 0 && g * N <= 32 && 32 % (g * N) == 0;
}

// Register budget of a variant: the floats a lane keeps live (gathered rows
// of a batch, local row, accumulator, gradient row) stay within 160.
template <int MODE, typename T>
constexpr bool fits_registers(int V, int U)
{
    const int E = V * (16 / (int)sizeof(T));
    const int rows = U * (MODE == M_BWD_COL ? 2 : 1) + 2 + (MODE == M_BWD_ROW ? 1 : 0);
    return E * rows <= 160;
}

// Minimum vectors per lane of a row shape (rows of more than 32 vectors
// need several per lane).
template <typename T, int R>
constexpr int base_vpl() { return (R * (int)sizeof(T) / 16) > 32 ? (R * (int)sizeof(T) / 16) / 32 : 1; }

template <int MODE, typename T, int R>
cudaError_t dispatch_variant(int vpl, int ng, int u, const PassArgs &a, cudaStream_t st)
{
    constexpr int B = base_vpl<T, R>();
#define FMM_TRY_VARIANT(V, N, UU)                                                   \
    if constexpr (team_ok<T, R>(V, N) && fits_registers<MODE, T>(V, UU)) {          \
        if (vpl == V && ng == N && u == UU)                                         \
            return launch_team<MODE, T, R, V, N, UU>(a, st);                        \
    }
    FMM_TRY_VARIANT(B, 1, 4)
    FMM_TRY_VARIANT(B, 1, 8)
    FMM_TRY_VARIANT(2 * B, 2, 2)
    FMM_TRY_VARIANT(2 * B, 2, 4)
    FMM_TRY_VARIANT(4 * B, 4, 1)
    FMM_TRY_VARIANT(4 * B, 4, 2)
    FMM_TRY_VARIANT(2 * B, 1, 4)
    FMM_TRY_VARIANT(B, 2, 4)
    FMM_TRY_VARIANT(B, 1, 2)
    FMM_TRY_VARIANT(B, 2, 2)
    FMM_TRY_VARIANT(2 * B, 1, 2)
    FMM_TRY_VARIANT(2 * B, 2, 1)
#undef FMM_TRY_VARIANT
    // a variant that does not fit this row shape: one group per row
    return launch_team<MODE, T, R, B, 1, 8>(a, st);
}

template <typename T, int R>
cudaError_t dispatch_mode(int mode, int vpl, int ng, int u, const PassArgs &a, cudaStream_t st)
{
    switch (mode) {
    case M_FUSED: return dispatch_variant<M_FUSED, T, R>(vpl, ng, u, a, st);
    case M_SDDMM: return dispatch_variant<M_SDDMM, T, R>(vpl, ng, u, a, st);
    case M_SPMM: return dispatch_variant<M_SPMM, T, R>(vpl, ng, u, a, st);
    case M_BWD_ROW: return dispatch_variant<M_BWD_ROW, T, R>(vpl, ng, u, a, st);
    case M_BWD_COL: return dispatch_variant<M_BWD_COL, T, R>(vpl, ng, u, a, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_generic(int mode, const PassArgs &a, cudaStream_t st)
{
    const long long total = (long long)a.n_chunks + a.n_light;
    const long long blocks = (total + 7) / 8;
    switch (mode) {
    case M_FUSED: row_pass_generic<M_FUSED, T><<<(unsigned)blocks, 256, 0, st>>>(a); break;
    case M_SDDMM: row_pass_generic<M_SDDMM, T><<<(unsigned)blocks, 256, 0, st>>>(a); break;
    case M_SPMM: row_pass_generic<M_SPMM, T><<<(unsigned)blocks, 256, 0, st>>>(a); break;
    case M_BWD_ROW: row_pass_generic<M_BWD_ROW, T><<<(unsigned)blocks, 256, 0, st>>>(a); break;
    case M_BWD_COL: row_pass_generic<M_BWD_COL, T><<<(unsigned)blocks, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// vpl is given in multiples of the shape's minimum (1, 2 or 4).
template <typename T>
cudaError_t launch_pass_typed(int mode, int vpl_mult, int ng, int u, bool vec, const PassArgs &a,
                              cudaStream_t st)
{
    const long long total = (long long)a.n_chunks + a.n_light;
    if (total == 0)
        return cudaSuccess;
    if (vec) {
        switch (a.r) {
        case 32: return dispatch_mode<T, 32>(mode, vpl_mult * base_vpl<T, 32>(), ng, u, a, st);
        case 64: return dispatch_mode<T, 64>(mode, vpl_mult * base_vpl<T, 64>(), ng, u, a, st);
        case 128: return dispatch_mode<T, 128>(mode, vpl_mult * base_vpl<T, 128>(), ng, u, a, st);
        case 256: return dispatch_mode<T, 256>(mode, vpl_mult * base_vpl<T, 256>(), ng, u, a, st);
        default: break;
        }
    }
    return launch_generic<T>(mode, a, st);
}

}  // namespace fmm
