// Streaming evaluation of the radix-2 sliding tree along one axis (arXiv 1707.08213,
// Section 4.2 Eqs. rowfswft2d / colfswft2d restricted to one dimension; Section 4.3's
// "trees innermost" loop order).
//
// A thread walks the window-end position p along the axis one step at a time.  For a
// window of n = 2^M samples the tree under p has levels v = 1..M; node i < 2^v of level v is
//
//     T_v(p)[i] = T_{v-1}(p - s_v)[i mod 2^(v-1)] + W_v^i * T_{v-1}(p)[i mod 2^(v-1)],
//     s_v = 2^(M-v),  W_v^i = Omega[i * s_v] = w_{2^v}^{-i},
//
// and level 0 is the data.  Nodes i and i + 2^(v-1) share both operands and W differs by a
// sign, so each pair is one butterfly: one complex multiply, one add, one subtract.
//
// GB300 mapping.  The level-(v-1) values a step needs from position p - s_v were computed
// by this same thread s_v steps earlier, so each level keeps a FIFO ("ring") of its last
// s_{v} = 2^(M-v) values.  Unrolling the step loop by the longest ring (2^(M-2) steps)
// makes every ring slot a compile-time register: no shared memory, no synchronisation.
// Level 0 needs no ring: T_0(p - n/2) is the input sample, re-read from memory (L1).
//
// Splitting one tree over 2^B threads: thread c keeps only the nodes i == c (mod 2^B) of
// every level >= B (their parents have the same residue), and the single node c mod 2^v
// of each level v < B.  The 2^B threads of a tree then need no communication; levels < B
// are repeated per thread (B - 1 extra node evaluations per step), which buys 2^B times
// the parallelism and divides the ring registers.  Thread c produces outputs
// k = c + 2^B t, t < 2^(M-B).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace swdft {

__host__ __device__ constexpr int tg_held(int B, int u) { return u <= B ? 1 : (1 << (u - B)); }
__host__ __device__ constexpr int tg_depth(int M, int u) { return 1 << (M - u - 1); }
__host__ __device__ constexpr int tg_off(int M, int B, int u) {
    int o = 0;
    for (int w = 1; w < u; ++w) o += tg_depth(M, w) * tg_held(B, w);
    return o;
}
__host__ __device__ constexpr int tg_ring(int M, int B) { return M >= 2 ? tg_off(M, B, M) : 0; }
__host__ __device__ constexpr int tg_period(int M) { return M >= 2 ? (1 << (M - 2)) : 1; }
__host__ __device__ constexpr int tg_twoff(int B, int v) {
    int t = 0;
    for (int w = 1; w < v; ++w) t += (w <= B) ? 1 : tg_held(B, w - 1);
    return t;
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 w, float2 d) {
    return make_float2(fmaf(w.x, d.x, -w.y * d.y), fmaf(w.x, d.y, w.y * d.x));
}
__device__ __forceinline__ float2 c_scale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

// One axis, window 2^M, nodes split over 2^B threads (B <= M).
template <int M, int B>
struct SlidingTree {
    static_assert(B >= 0 && B <= M, "residue split larger than the tree");
    static constexpr int kN = 1 << M;
    static constexpr int kRing = tg_ring(M, B);
    static constexpr int kTw = tg_twoff(B, M + 1);
    static constexpr int kOut = tg_held(B, M);    // outputs per step
    static constexpr int kPeriod = tg_period(M);  // steps per unrolled group
    static constexpr int kHalf = kN / 2;          // level-0 look-back of level 1

    float2 ring[kRing > 0 ? kRing : 1];
    float2 tw[kTw > 0 ? kTw : 1];

    // c: this thread's residue (< 2^B); om64: Omega of length 64, om64[j] = w_64^{-j}.
    // W_v^i = w_{2^v}^{-i} = om64[i * 2^(6-v)], the same FP32 value as Omega^(2^M)[i * s_v].
    __device__ __forceinline__ void init(int c, const float2 *om64) {
        static_assert(M <= 6, "twiddle table covers windows up to 64");
        const int cb = c & ((1 << B) - 1);
#pragma unroll
        for (int v = 1; v <= M; ++v) {
            const int base = tg_twoff(B, v);
            if (v <= B) {
                const int i = c & ((1 << v) - 1);
                tw[base] = om64[i << (6 - v)];
            } else {
#pragma unroll
                for (int t = 0; t < tg_held(B, v - 1); ++t) tw[base + t] = om64[(cb + (t << B)) << (6 - v)];
            }
        }
#pragma unroll
        for (int i = 0; i < (kRing > 0 ? kRing : 1); ++i) ring[i] = make_float2(0.f, 0.f);
    }

    // Step J (mod kPeriod): x_p = level 0 at p, x_s = level 0 at p - n/2.
    // out[t] = level-M node c + 2^B t at p.
    template <int J>
    __device__ __forceinline__ void step(float2 x_p, float2 x_s, float2 (&out)[kOut]) {
        out[0] = x_p;
        level<J, 1>(out, x_s);
    }

  private:
    template <int J, int V>
    __device__ __forceinline__ void level(float2 (&cur)[kOut], float2 x_s) {
        if constexpr (V <= M) {
            constexpr int Hp = tg_held(B, V - 1);
            float2 old[Hp];
            if constexpr (V == 1) {
                old[0] = x_s;
            } else {
                // FIFO of level V-1, depth s_V = 2^(M-V): read the value from p - s_V, then
                // store the value at p in the same slot.
                constexpr int D = tg_depth(M, V - 1);
                constexpr int base = tg_off(M, B, V - 1) + (J % D) * Hp;
#pragma unroll
                for (int t = 0; t < Hp; ++t) {
                    old[t] = ring[base + t];
                    ring[base + t] = cur[t];
                }
            }
            constexpr int tb = tg_twoff(B, V);
            if constexpr (V <= B) {
                cur[0] = c_add(old[0], c_mul(tw[tb], cur[0]));
            } else {
#pragma unroll
                for (int t = 0; t < Hp; ++t) {
                    const float2 p = c_mul(tw[tb + t], cur[t]);
                    cur[t + Hp] = c_sub(old[t], p);
                    cur[t] = c_add(old[t], p);
                }
            }
            level<J, V + 1>(cur, x_s);
        }
    }
};

}  // namespace swdft
