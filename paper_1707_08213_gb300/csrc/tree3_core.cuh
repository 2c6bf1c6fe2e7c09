// Streaming ternary sliding tree: windows of 3^M samples (M <= 3) along one axis.
//
// The paper (arXiv 1707.08213) derives binary trees (Section 4.2) and notes that radix 3
// replaces them by ternary ones (Section 5).  Level t (t = 1..M) of the tree under
// position p holds the 3^t-point DFT of the samples spaced s_t = 3^(M-t) apart that end at
// p; they interleave three 3^(t-1)-point sequences ending at p - 2 s_t, p - s_t and p, so
//
//     T_t(p)[i' + k 3^(t-1)] = sum_{d<3} w_3^{-k d} w_{3^t}^{-i' d} T_(t-1)(p - (2-d) s_t)[i'],
//
// i' < 3^(t-1), k < 3: per i' one radix-3 butterfly on the inputs twiddled by w_{3^t}^{-i' d}.
// Level 0 is the data; level M is the window's DFT in natural order.
//
// GB300 mapping, as for the binary tree (tree_core.cuh): a thread walks positions and keeps
// the level values it needs later in register FIFOs.  Level t reads level t-1 from s_t and
// 2 s_t steps back, so level t-1 keeps a FIFO of 2 s_t slots; unrolling the walk by
// 2 s_2 = 2 * 3^(M-2) steps (every FIFO depth divides it) makes each slot a compile-time
// register.  Level 0's look-backs (p - s_1, p - 2 s_1) are re-read from memory (shared
// memory in the column pass).  Three threads share a tree, one per node residue mod 3.
#pragma once

#include "swdft_internal.h"
#include "tree_core.cuh"

namespace swdft {

__host__ __device__ constexpr int pow3(int m) { return m <= 0 ? 1 : 3 * pow3(m - 1); }

// w_27^{-j}, j < 27 (FP64-evaluated, FP32-rounded): every 3^m <= 27 is its strided view.
// h = sin(pi/3) from the same table (-Im w_27^{-9}), for the radix-3 butterfly.
struct Omega27 {
    float2 w[kMaxN3];
    float h;
};

// Y0 = B0 + B1 + B2, Y1 = B0 + w3^-1 B1 + w3^-2 B2, Y2 = B0 + w3^-2 B1 + w3^-1 B2,
// w3^-1 = -1/2 - i h, w3^-2 = -1/2 + i h.
__device__ __forceinline__ void bfly3(float2 b0, float2 b1, float2 b2, float h, float2 &y0, float2 &y1,
                                      float2 &y2) {
    const float2 s = c_add(b1, b2);
    const float2 d = c_sub(b1, b2);
    const float2 t = make_float2(fmaf(-0.5f, s.x, b0.x), fmaf(-0.5f, s.y, b0.y));
    const float2 u = make_float2(h * d.y, -h * d.x);  // -i h d
    y0 = c_add(b0, s);
    y1 = c_add(t, u);
    y2 = c_sub(t, u);
}

// The tree split over three threads by node residue (M >= 1).  For t >= 2 a level-t
// node i is computed from level-(t-1) node i mod 3^(t-1), which has the same residue mod 3,
// so thread c (< 3) keeps only the nodes == c (mod 3) of every level: level 1's node c
// (a three-term sum), then at level t the 3^(t-2) butterflies on i' == c (mod 3).  No data
// passes between the three threads and no node is evaluated twice.  Thread c produces the
// outputs k = c + 3 u, u < 3^(M-1), in that order.
template <int M>
struct SlidingTree3Split {
    static_assert(M >= 1 && M <= kMaxLog3, "split ternary trees: windows 3, 9, 27");
    static constexpr int kN = pow3(M);
    static constexpr int kOut = pow3(M - 1);  // outputs per thread
    static constexpr int kPeriod = M >= 2 ? 2 * pow3(M - 2) : 1;
    static constexpr int kS1 = pow3(M - 1);
    // FIFO of level t-1 (t >= 2): depth 2 s_t slots of 3^(t-2) values (nodes == c mod 3)
    static constexpr int held(int t) { return t <= 1 ? 1 : pow3(t - 1); }  // level-t nodes held
    static constexpr int fifo_off(int t) {
        int o = 0;
        for (int u = 2; u < t; ++u) o += 2 * pow3(M - u) * held(u - 1);
        return o;
    }
    static constexpr int kFifo = M >= 2 ? fifo_off(M + 1) : 0;
    // twiddles: level 1: w_3^{-c}, w_3^{-2c}; level t >= 2: w_{3^t}^{-i'}, w_{3^t}^{-2 i'} for
    // each i' = c + 3 a, a < 3^(t-2)
    static constexpr int tw_off(int t) {
        int o = 2;
        for (int u = 2; u < t; ++u) o += 2 * pow3(u - 2);
        return o;
    }
    static constexpr int kTw = tw_off(M + 1);

    float2 fifo[kFifo > 0 ? kFifo : 1];
    float2 tw[kTw];

    __device__ __forceinline__ void init(int c, const Omega27 &om) {
        tw[0] = om.w[(9 * c) % kMaxN3];
        tw[1] = om.w[(18 * c) % kMaxN3];
        static_for<2, M + 1>([&](auto TT) {
            constexpr int t = decltype(TT)::value;
            constexpr int step = kMaxN3 / pow3(t);
            static_for<0, pow3(t - 2)>([&](auto AA) {
                constexpr int a = decltype(AA)::value;
                const int ip = c + 3 * a;
                tw[tw_off(t) + 2 * a] = om.w[(ip * step) % kMaxN3];
                tw[tw_off(t) + 2 * a + 1] = om.w[(2 * ip * step) % kMaxN3];
            });
        });
#pragma unroll
        for (int i = 0; i < (kFifo > 0 ? kFifo : 1); ++i) fifo[i] = make_float2(0.f, 0.f);
    }

    // out[u] = level-M node c + 3 u at p.
    template <int J>
    __device__ __forceinline__ void step(float h, float2 x_p, float2 x_s1, float2 x_s2, float2 (&out)[kOut]) {
        // level 1, node c: x(p - 2 s1) + w_3^{-c} x(p - s1) + w_3^{-2c} x(p)
        float2 cur[kOut];
        cur[0] = c_add(x_s2, c_add(c_mul(tw[0], x_s1), c_mul(tw[1], x_p)));
        level<J, 2>(h, cur);
#pragma unroll
        for (int u = 0; u < kOut; ++u) out[u] = cur[u];
    }

  private:
    // cur holds level T-1's nodes c + 3 a (a < held(T-1)) in slots a; on return level T's
    // nodes c + 3 a' (a' < held(T)) in slots a'.
    template <int J, int T>
    __device__ __forceinline__ void level(float h, float2 (&cur)[kOut]) {
        if constexpr (T <= M) {
            constexpr int s = pow3(M - T);
            constexpr int D = 2 * s;
            constexpr int HP = held(T - 1);        // level T-1 nodes held = butterflies here
            constexpr int off = fifo_off(T);
            constexpr int now = (J % D) * HP;
            constexpr int back1 = ((J + s) % D) * HP;
            constexpr int tb = tw_off(T);
            float2 nxt[kOut];
#pragma unroll
            for (int a = 0; a < HP; ++a) {
                // node i' = c + 3 a of level T-1 (or node c of level 1 when T = 2)
                const float2 a2 = cur[a];
                const float2 a1 = fifo[off + back1 + a];
                const float2 a0 = fifo[off + now + a];
                fifo[off + now + a] = a2;
                const float2 b1 = c_mul(tw[tb + 2 * a], a1);
                const float2 b2 = c_mul(tw[tb + 2 * a + 1], a2);
                // outputs i' + k 3^(T-1) = c + 3 (a + k 3^(T-2)): slots a + k * HP
                bfly3(a0, b1, b2, h, nxt[a], nxt[a + HP], nxt[a + 2 * HP]);
            }
#pragma unroll
            for (int a = 0; a < 3 * HP; ++a) cur[a] = nxt[a];
            level<J, T + 1>(h, cur);
        }
    }
};

}  // namespace swdft
