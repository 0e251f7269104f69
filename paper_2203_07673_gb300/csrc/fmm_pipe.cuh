// Pipelined row pass: the gathered rows of the next batches are already in
// flight while the current batch is used.
//
// The team kernel (fmm_rows.cuh) issues the gathers of a batch and then
// waits for them, so a team has at most one batch of rows in flight and its
// warp idles for the whole load latency once per batch.  On patterns whose
// gathers mostly hit L2 with short dense rows (bfloat16 rows of r = 64,
// 128 bytes) that wait, not bandwidth, sets the pass time.  Here a team keeps
// a ring of RING batches of gathered rows in registers, as the raw 16-byte
// words (bfloat16 rows stay packed until used).  Two orders: REFILL = 0
// issues the loads of batch b + RING - 1 into the slot freed by batch b - 1
// and then uses batch b; REFILL = 1 reads batch b out of its slot, refills
// that slot at once with batch b + RING and then uses batch b (one batch
// further ahead for the same registers).  The ring is indexed
// with compile-time slots only (the loop over one index block is fully
// unrolled), so it stays in registers.
//
// Arithmetic uses the paired float32 instructions (__ffma2_rn, __fadd2_rn:
// two round-to-nearest operations in one instruction): the partial dot
// product of a lane runs as two interleaved chains (even and odd elements)
// summed at the end, the accumulation updates two elements per instruction,
// and the U dot products of a batch are reduced across the lane group in
// pairs.
//
// Column indices and values come in index blocks of IB nonzeros (K per
// lane, coalesced) handed out by shuffles; the current and the next block
// are held, which covers a prefetch distance of up to one block.  Nonzeros
// past the end of a row get value 0 and a zero row, so every batch runs the
// same instructions and contributes exactly nothing.
//
// Row layout: with two or more 16-byte words per lane, a lane owns
// consecutive words of a row (lane l: words l VPL ... l VPL + VPL - 1), so a
// gathered row reaches the lane in 32-byte loads (ld.global.nc.v8.b32) and
// each load instruction of the warp touches one 128-byte line per bfloat16
// row of r = 64, where word-interleaved 16-byte loads touch every line twice.
// The gathered operand must be 32-byte aligned.
//
// Roles: FusedMM, SDDMM, SpMM, and the two adjoint passes: over S (two
// dot products of the gathered row, against the local row and the local
// float32 gradient row; ds written) and over S^T (the gathered row and its
// float32 gradient row both in the ring).  The pass over S is instantiated
// for the default layout only (code 32212): on R-MAT 2^22 with bfloat16 rows
// of r = 64 the backward took 5.205 ms with it against 5.289 ms with the
// team kernel; the pass over S^T (5.47 ms with it) is not instantiated.  One
// team of G lanes per row or chunk of a split row.
#pragma once

#include "fmm_rows.cuh"

namespace fmm {

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Two consecutive 16-byte words of a row from a 32-byte-aligned address, by
// one 32-byte load on the read-only path.
__device__ __forceinline__ void load32(const void *p, uint4 &w0, uint4 &w1)
{
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w0.x), "=r"(w0.y), "=r"(w0.z), "=r"(w0.w), "=r"(w1.x), "=r"(w1.y),
                   "=r"(w1.z), "=r"(w1.w)
                 : "l"(p));
}

// The 16-byte word q of a row of T as float pairs (element 2i, 2i + 1).
template <typename T>
__device__ __forceinline__ void unpack2(const uint4 q, float2 *f)
{
    if constexpr (sizeof(T) == 2) {
        f[0] = make_float2(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u));
        f[1] = make_float2(__uint_as_float(q.y << 16), __uint_as_float(q.y & 0xffff0000u));
        f[2] = make_float2(__uint_as_float(q.z << 16), __uint_as_float(q.z & 0xffff0000u));
        f[3] = make_float2(__uint_as_float(q.w << 16), __uint_as_float(q.w & 0xffff0000u));
    } else {
        f[0] = make_float2(__uint_as_float(q.x), __uint_as_float(q.y));
        f[1] = make_float2(__uint_as_float(q.z), __uint_as_float(q.w));
    }
}

// Blocks of one warp: a block retires when its slowest row is done, so
// small blocks let the SM start new rows as soon as a warp is free (GB300,
// against 256-thread blocks: FusedMMA on Zipf rows 1.341 -> 1.294 ms, R-MAT
// forward 1.416 -> 1.345 ms; 64-thread blocks 1.302 / 1.352).
constexpr int kPipeBlock = 32;

// MB is the number of 256 threads a variant asks to keep resident per SM,
// as 256 / kPipeBlock blocks each (a register cap of 65536 / (256 MB) per
// thread): the register ring trades rows in flight per team against teams
// per SM.
template <int MODE, typename T, int R, int VPL, int U, int RING, int MB, int REFILL>
__global__ void __launch_bounds__(kPipeBlock, MB * (256 / kPipeBlock)) pipe_pass_kernel(const PassArgs a)
{
    static_assert(MODE >= M_FUSED && MODE <= M_BWD_COL, "role");
    using TS = TeamShape<T, R, VPL, 1>;
    constexpr int G = TS::G, E = TS::E, EPV = TS::EPV;
    constexpr int E2 = E / 2, W2 = EPV / 2;   // float pairs per lane; per 16-byte word
    constexpr int K = G >= 8 ? 1 : 8 / G;     // index entries per lane per block
    constexpr int IB = K * G;                 // nonzeros per index block
    constexpr int BPB = IB / U;               // batches per index block
    static_assert(IB % U == 0 && BPB % RING == 0 && RING >= 2 - REFILL, "ring layout");
    constexpr bool HAS_L = MODE != M_SPMM;
    constexpr bool ACC = MODE != M_SDDMM;
    constexpr bool NZ = MODE == M_SDDMM || MODE == M_BWD_ROW;
    constexpr bool TWO = MODE == M_BWD_ROW || MODE == M_BWD_COL;   // two dot products
    constexpr bool LOCAL_H = MODE == M_BWD_ROW;    // float32 gradient row, local
    constexpr bool GATHER_H = MODE == M_BWD_COL;   // float32 gradient row, gathered
    constexpr int HW = GATHER_H ? VPL * EPV / 4 : 1;   // float4 words of a gathered H row
    constexpr int ND = TWO ? 2 * U : U;                // dot products per batch
    constexpr bool WIDE = VPL % 2 == 0;                // lane-contiguous words, 32-byte loads

    const int lane = threadIdx.x & 31;
    const int lig = lane & (G - 1);
    const int tbase = lane & ~(G - 1);
    // the row word that word v of this lane holds
    auto widx = [lig](int v) { return WIDE ? lig * VPL + v : v * G + lig; };
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const long long total = (long long)a.n_chunks + a.n_light;
    const bool active = gid < total;
    const Loader ld;

    int row = 0, beg = 0, end = 0, slot = -1;
    if (active)
        pass_item(a, gid, row, beg, end, slot);
    const T *L = static_cast<const T *>(a.L);
    const T *Y = static_cast<const T *>(a.Y);

    float2 l2[E2], acc2[E2], h2[LOCAL_H ? E2 : 1];
#pragma unroll
    for (int e = 0; e < E2; ++e) {
        l2[e] = make_float2(0.f, 0.f);
        acc2[e] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < (LOCAL_H ? E2 : 1); ++e)
        h2[e] = make_float2(0.f, 0.f);   // rows without nonzeros never load theirs
    // a float32 row in T's element mapping (word v of the lane holds EPV
    // elements): EPV / 4 float4 per word
    auto load_h = [&](const float *hrow, float2 *f, bool gather) {
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int q = 0; q < EPV / 4; ++q) {
                const float4 x = ld.f4(hrow + widx(v) * EPV + 4 * q, gather);
                f[v * W2 + 2 * q] = make_float2(x.x, x.y);
                f[v * W2 + 2 * q + 1] = make_float2(x.z, x.w);
            }
    };
    if constexpr (LOCAL_H)
        if (active && end > beg)
            load_h(a.H + (size_t)row * R, h2, false);
    if (HAS_L && active && end > beg) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const uint4 q = ld.u4(reinterpret_cast<const uint4 *>(L + (size_t)row * R) + widx(v),
                                  false);
            unpack2<T>(q, &l2[v * W2]);
        }
    }

    const int n = end - beg;
    const int wn = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
    const int wblocks = (wn + IB - 1) / IB;

    // index block b: entry e of lane l is nonzero b * IB + e * G + l; past
    // the end of the row j = -1 and s = 0
    int jc[K], jn[K], ic[K], in_[K];
    float sc[K], sn[K];
    // per-nonzero outputs (SDDMM): the lane holding a nonzero's index entry
    // keeps its value and stores the block's values at once
    float held[K];
#pragma unroll
    for (int e = 0; e < K; ++e) held[e] = 0.f;
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

    uint4 ring[RING][U][VPL];
    float4 hring[GATHER_H ? RING : 1][U][HW];

    // gathers of batch bb (block-local) of the block whose indices are j
    auto issue = [&](uint4 (&dst)[U][VPL], const int (&j)[K], int bb) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = bb * U + u;
            const int jj = __shfl_sync(0xffffffffu, j[t / G], tbase + (t % G));
            if constexpr (WIDE) {
#pragma unroll
                for (int v = 0; v < VPL; v += 2) {
                    dst[u][v] = make_uint4(0u, 0u, 0u, 0u);
                    dst[u][v + 1] = make_uint4(0u, 0u, 0u, 0u);
                    if (jj >= 0)
                        load32(reinterpret_cast<const uint4 *>(Y + (size_t)jj * R) + widx(v),
                               dst[u][v], dst[u][v + 1]);
                }
            } else {
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    dst[u][v] = make_uint4(0u, 0u, 0u, 0u);
                    if (jj >= 0)
                        dst[u][v] = ld.u4(reinterpret_cast<const uint4 *>(Y + (size_t)jj * R) + widx(v),
                                          true);
                }
            }
        }
    };
    // the gathered float32 gradient rows of the same batch
    auto issue_h = [&](float4 (&dst)[U][HW], const int (&j)[K], int bb) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = bb * U + u;
            const int jj = __shfl_sync(0xffffffffu, j[t / G], tbase + (t % G));
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int q = 0; q < EPV / 4; ++q) {
                    dst[u][v * (EPV / 4) + q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (jj >= 0)
                        dst[u][v * (EPV / 4) + q] =
                            ld.f4(a.H + (size_t)jj * R + widx(v) * EPV + 4 * q, true);
                }
        }
    };
    auto issue_all = [&](int slot_, const int (&j)[K], int bb) {
        issue(ring[slot_], j, bb);
        if constexpr (GATHER_H)
            issue_h(hring[slot_], j, bb);
    };

    load_block(0, jc, sc, ic);
    load_block(1, jn, sn, in_);
#pragma unroll
    for (int b = 0; b < RING - 1 + REFILL; ++b)
        issue_all(b, jc, b);

    for (int bk = 0; bk < wblocks; ++bk) {
#pragma unroll
        for (int bb = 0; bb < BPB; ++bb) {
            if constexpr (!REFILL) {
                // batch bb + RING - 1 into the slot that batch bb - 1 freed
                const int pf = bb + RING - 1;
                if (pf < BPB)
                    issue_all(pf % RING, jc, pf);
                else
                    issue_all(pf % RING, jn, pf - BPB);
            }
            // use batch bb
            float sv[U];
            int sidx[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = bb * U + u;
                sv[u] = __shfl_sync(0xffffffffu, sc[t / G], tbase + (t % G));
                sidx[u] = (NZ && MODE != M_SDDMM) ? __shfl_sync(0xffffffffu, ic[t / G], tbase + (t % G))
                                                  : 0;
            }
            float2 y2[U][E2];
            float2 g2[GATHER_H ? U : 1][GATHER_H ? E2 : 1];
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int v = 0; v < VPL; ++v)
                    unpack2<T>(ring[bb % RING][u][v], &y2[u][v * W2]);
                if constexpr (GATHER_H) {
#pragma unroll
                    for (int q = 0; q < HW; ++q) {
                        const float4 x = hring[bb % RING][u][q];
                        g2[u][2 * q] = make_float2(x.x, x.y);
                        g2[u][2 * q + 1] = make_float2(x.z, x.w);
                    }
                }
            }
            // the slot just read takes batch bb + RING (RING batches ahead;
            // batches past this block come from the next index block)
            if constexpr (REFILL) {
                const int pf = bb + RING;
                if (pf < BPB)
                    issue_all(bb % RING, jc, pf);
                else
                    issue_all(bb % RING, jn, pf - BPB);
            }
            if constexpr (MODE == M_SPMM) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float2 c2 = make_float2(sv[u], sv[u]);
#pragma unroll
                    for (int e = 0; e < E2; ++e)
                        acc2[e] = ffma2(c2, y2[u][e], acc2[e]);
                }
            } else {
                // d[u] = <L, Y_u>; with two dot products d[U + u] = <H, Y_u>
                // (over S) or <H_u, L> (over S^T)
                float d[ND];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    float2 t2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int e = 0; e < E2; ++e)
                        t2 = ffma2(l2[e], y2[u][e], t2);
                    d[u] = t2.x + t2.y;
                    if constexpr (TWO) {
                        float2 w2 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int e = 0; e < E2; ++e) {
                            if constexpr (LOCAL_H)
                                w2 = ffma2(h2[e], y2[u][e], w2);
                            else
                                w2 = ffma2(g2[u][e], l2[e], w2);
                        }
                        d[U + u] = w2.x + w2.y;
                    }
                }
                // sum over the G lanes of the group, two dot products per step
#pragma unroll
                for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
                    for (int i = 0; i + 1 < ND; i += 2) {
                        const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, d[i], off),
                                                     __shfl_xor_sync(0xffffffffu, d[i + 1], off));
                        const float2 s2 = fadd2(make_float2(d[i], d[i + 1]), o);
                        d[i] = s2.x;
                        d[i + 1] = s2.y;
                    }
                    if constexpr (ND % 2)
                        d[ND - 1] += __shfl_xor_sync(0xffffffffu, d[ND - 1], off);
                }
                if constexpr (MODE == M_FUSED) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float c = sv[u] * d[u];
                        const float2 c2 = make_float2(c, c);
#pragma unroll
                        for (int e = 0; e < E2; ++e)
                            acc2[e] = ffma2(c2, y2[u][e], acc2[e]);
                    }
                } else if constexpr (MODE == M_SDDMM) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int t = bb * U + u;
                        if (lig == t % G)
                            held[t / G] = sv[u] * d[u];
                    }
                } else if constexpr (MODE == M_BWD_ROW) {
                    // ds = <A_i, B_j> <G_i, B_j>;  dA_i += s <G_i, B_j> B_j
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (a.nzout && sidx[u] >= 0 && lig == (u % G))
                            a.nzout[sidx[u]] = d[u] * d[U + u];
                        const float c = sv[u] * d[U + u];
                        const float2 c2 = make_float2(c, c);
#pragma unroll
                        for (int e = 0; e < E2; ++e)
                            acc2[e] = ffma2(c2, y2[u][e], acc2[e]);
                    }
                } else {   // M_BWD_COL: dB_j += s (<A_i, B_j> G_i + <G_i, B_j> A_i)
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float c1 = sv[u] * d[u], c2s = sv[u] * d[U + u];
                        const float2 c1v = make_float2(c1, c1), c2v = make_float2(c2s, c2s);
#pragma unroll
                        for (int e = 0; e < E2; ++e)
                            acc2[e] = ffma2(c1v, g2[u][e], ffma2(c2v, y2[u][e], acc2[e]));
                    }
                }
            }
        }
        if constexpr (MODE == M_SDDMM) {
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

    if constexpr (ACC) {
        if (active) {
            float *dst = slot >= 0 ? a.partials + (size_t)slot * R
                                   : (a.out ? a.out + (size_t)row * R : nullptr);
            if (dst) {
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
#pragma unroll
                    for (int w = 0; w < W2; w += 2) {
                        const int k = widx(v) * EPV + 2 * w;
                        const float2 p0 = acc2[v * W2 + w], p1 = acc2[v * W2 + w + 1];
                        out_store4(ld, dst + k, make_float4(p0.x, p0.y, p1.x, p1.y),
                                   a.accumulate && slot < 0);
                    }
                }
            }
        }
    }
}

template <int MODE, typename T, int R, int VPL, int U, int RING, int MB, int REFILL>
cudaError_t launch_pipe(const PassArgs &a, cudaStream_t st)
{
    constexpr int G = TeamShape<T, R, VPL, 1>::G;
    const long long total = (long long)a.n_chunks + a.n_light;
    const long long blocks = (total * G + kPipeBlock - 1) / kPipeBlock;
    pipe_pass_kernel<MODE, T, R, VPL, U, RING, MB, REFILL><<<(unsigned)blocks, kPipeBlock, 0, st>>>(a);
    return cudaGetLastError();
}

// Whether (VPL, U, RING) fits rows of R elements of T: a valid team layout
// whose index block holds a whole number of rings of batches.
template <typename T, int R>
constexpr bool pipe_ok(int V, int U, int RING)
{
    if (!team_ok<T, R>(V, 1))
        return false;
    const int g = R * (int)sizeof(T) / 16 / V;
    const int ib = (g >= 8 ? 1 : 8 / g) * g;
    return ib % (U * RING) == 0;
}

// Variants: (VPL, U, RING, MB, REFILL) with VPL as a multiple of the row
// shape's minimum.
template <typename T, int R>
cudaError_t dispatch_pipe(int mode, int vpl, int u, int ring, int mb, int refill,
                          const PassArgs &a, cudaStream_t st)
{
    constexpr int B = base_vpl<T, R>();
#define FMM_PIPE(M, V, UU, RR, MM, FF)                                             \
    if constexpr (pipe_ok<T, R>(V, UU, RR))                                        \
        if (mode == M && vpl == V && u == UU && ring == RR && mb == MM && refill == FF) \
            return launch_pipe<M, T, R, V, UU, RR, MM, FF>(a, st);
#define FMM_PIPE_MODES(V, UU, RR, MM, FF)                                         \
    FMM_PIPE(M_FUSED, V, UU, RR, MM, FF) FMM_PIPE(M_SDDMM, V, UU, RR, MM, FF)       \
    FMM_PIPE(M_SPMM, V, UU, RR, MM, FF)
    FMM_PIPE_MODES(2 * B, 1, 2, 2, 0)
    FMM_PIPE_MODES(2 * B, 1, 2, 3, 0)
    FMM_PIPE_MODES(2 * B, 1, 4, 2, 0)
    FMM_PIPE_MODES(2 * B, 1, 2, 2, 1) FMM_PIPE(M_BWD_ROW, 2 * B, 1, 2, 2, 1)
    FMM_PIPE_MODES(B, 2, 2, 4, 0)
    FMM_PIPE_MODES(B, 2, 2, 4, 1)
    FMM_PIPE_MODES(B, 2, 4, 3, 0)
    FMM_PIPE_MODES(B, 4, 2, 3, 0)
#undef FMM_PIPE_MODES
#undef FMM_PIPE
    return cudaErrorNotSupported;   // not instantiated for this width: the caller falls back
}

template <typename T>
cudaError_t launch_pipe_typed(int mode, int vpl_mult, int u, int ring, int mb, int refill,
                              const PassArgs &a, cudaStream_t st)
{
    if ((long long)a.n_chunks + a.n_light == 0)
        return cudaSuccess;
    switch (a.r) {
    case 32: return dispatch_pipe<T, 32>(mode, vpl_mult * base_vpl<T, 32>(), u, ring, mb, refill, a, st);
    case 64: return dispatch_pipe<T, 64>(mode, vpl_mult * base_vpl<T, 64>(), u, ring, mb, refill, a, st);
    case 128: return dispatch_pipe<T, 128>(mode, vpl_mult * base_vpl<T, 128>(), u, ring, mb, refill, a, st);
    case 256: return dispatch_pipe<T, 256>(mode, vpl_mult * base_vpl<T, 256>(), u, ring, mb, refill, a, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace fmm
