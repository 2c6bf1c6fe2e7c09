// Adjoint of the streaming sliding tree (see tree_core.cuh): the transposed butterfly
// graph of arXiv 1707.08213 Section 4.2 along one axis, walked with decreasing position.
#pragma once

#include "tree_core.cuh"

namespace swdft {

// ------------------------------------------------------------------------------------
// Adjoint of SlidingTree: the transposed butterfly graph, walked with decreasing p.
//
// The forward map sends a 1D sequence x to every window's DFT; its adjoint sends per-window
// spectra G[q][k] to y[p] = sum_j sum_k G[p-j][k] w_n^{+jk}: the overlap-add of every window's
// (unnormalised) inverse DFT.  Transposing the tree, with U_v(p) the adjoint of T_v(p):
//
//     U_{v-1}(p)[j] = conj(W_v^j) (U_v(p)[j] - U_v(p)[j+h]) + (U_v(p+s_v)[j] + U_v(p+s_v)[j+h]),
//
// h = 2^(v-1), U_M(p) = G[p-(n-1)] (0 where no window ends at p), y(p) = U_0(p)[0].  Only the
// pair sums of level v are needed s_v = 2^(M-v) steps later, so each level keeps a FIFO of
// n/2 pair sums, the same register budget as the forward tree; unrolled by the longest FIFO
// (level 1, 2^(M-1) steps).  Split over 2^B threads by residue: levels >= B need nothing from
// other threads; below B each thread carries its own partial of the single node it touches,
// and y(p) is the sum of the 2^B partials (reduced by the caller).
// ------------------------------------------------------------------------------------

// w * d + a: two fused multiply-adds per component
__device__ __forceinline__ float2 c_fma(float2 w, float2 d, float2 a) {
    return make_float2(fmaf(w.x, d.x, fmaf(-w.y, d.y, a.x)), fmaf(w.x, d.y, fmaf(w.y, d.x, a.y)));
}

__host__ __device__ constexpr int ta_slots(int B, int v) { return v > B ? tg_held(B, v - 1) : 1; }
__host__ __device__ constexpr int ta_off(int M, int B, int v) {
    // rings are laid out from level M down to level 1
    int o = 0;
    for (int w = M; w > v; --w) o += (1 << (M - w)) * ta_slots(B, w);
    return o;
}

template <int M, int B>
struct SlidingTreeAdjoint {
    static_assert(B >= 0 && B <= M, "residue split larger than the tree");
    static constexpr int kN = 1 << M;
    static constexpr int kIn = tg_held(B, M);                   // U_M nodes held
    static constexpr int kRing = M >= 1 ? ta_off(M, B, 0) : 0;
    static constexpr int kTw = tg_twoff(B, M + 1);
    static constexpr int kPeriod = M >= 1 ? (1 << (M - 1)) : 1;

    float2 ring[kRing > 0 ? kRing : 1];
    float2 tw[kTw > 0 ? kTw : 1];  // conjugated twiddles, same indexing as SlidingTree

    // om64[j] = w_64^{-j}; conj(W_v^i) = conj(om64[i * 2^(6-v)])
    __device__ __forceinline__ void init(int c, const float2 *om64) {
        static_assert(M <= 6, "twiddle table covers windows up to 64");
        const int cb = c & ((1 << B) - 1);
#pragma unroll
        for (int v = 1; v <= M; ++v) {
            const int base = tg_twoff(B, v);
            if (v <= B) {
                const float2 w = om64[(c & ((1 << v) - 1)) << (6 - v)];
                tw[base] = make_float2(w.x, -w.y);
            } else {
#pragma unroll
                for (int t = 0; t < tg_held(B, v - 1); ++t) {
                    const float2 w = om64[(cb + (t << B)) << (6 - v)];
                    tw[base + t] = make_float2(w.x, -w.y);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < (kRing > 0 ? kRing : 1); ++i) ring[i] = make_float2(0.f, 0.f);
    }

    // Step J (mod kPeriod) at position p: u = this thread's U_M(p) nodes (k = c + 2^B t);
    // returns this thread's partial of y(p).
    template <int J>
    __device__ __forceinline__ float2 step(float2 (&u)[kIn]) {
        level<J, M>(u);
        return u[0];
    }

    // Step J's partial of y(p) when this thread's level-1 node at p is zero: the level-1 FIFO
    // slot alone (U_1(p + s_1)'s pair sum, or below the split this thread's own partial), with
    // no level evaluated.  That holds at the last n/2 positions of a walk whose inputs stop
    // n - 1 steps before its end: U_1(p) depends on the inputs at p .. p + n/2 - 1 only.
    template <int J>
    __device__ __forceinline__ float2 tail() const {
        static_assert(M >= 1, "a window of one sample has no tree");
        return ring[ta_off(M, B, 1) + (J % (1 << (M - 1))) * ta_slots(B, 1)];
    }

  private:
    template <int J, int V>
    __device__ __forceinline__ void level(float2 (&cur)[kIn]) {
        if constexpr (V >= 1) {
            constexpr int D = 1 << (M - V);
            constexpr int base = ta_off(M, B, V) + (J % D) * ta_slots(B, V);
            constexpr int tb = tg_twoff(B, V);
            if constexpr (V > B) {
                constexpr int Hp = tg_held(B, V - 1);
#pragma unroll
                for (int t = 0; t < Hp; ++t) {
                    const float2 d = c_sub(cur[t], cur[t + Hp]);
                    const float2 s = c_add(cur[t], cur[t + Hp]);
                    const float2 old = ring[base + t];
                    ring[base + t] = s;
                    cur[t] = c_fma(tw[tb + t], d, old);
                }
            } else {
                const float2 old = ring[base];
                ring[base] = cur[0];
                cur[0] = c_fma(tw[tb], cur[0], old);
            }
            level<J, V - 1>(cur);
        }
    }
};

}  // namespace swdft
