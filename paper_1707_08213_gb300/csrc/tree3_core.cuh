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
// register.  Level 0's look-backs (p - s_1, p - 2 s_1) are re-read from memory.  One thread
// holds every node of its tree (3^B threads would not tile a warp), so every twiddle index
// is a compile-time constant and the twiddles are read straight from the kernel parameters.
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

template <int M>
struct SlidingTree3 {
    static_assert(M >= 0 && M <= kMaxLog3, "ternary windows up to 27");
    static constexpr int kN = pow3(M);
    static constexpr int kPeriod = M >= 2 ? 2 * pow3(M - 2) : 1;
    static constexpr int kS1 = M >= 1 ? pow3(M - 1) : 0;  // level-0 look-backs p - s1, p - 2 s1
    static constexpr int fifo_off(int t) {
        int o = 0;
        for (int u = 2; u < t; ++u) o += 2 * pow3(M - u) * pow3(u - 1);
        return o;
    }
    static constexpr int kFifo = M >= 2 ? fifo_off(M + 1) : 0;

    float2 fifo[kFifo > 0 ? kFifo : 1];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < (kFifo > 0 ? kFifo : 1); ++i) fifo[i] = make_float2(0.f, 0.f);
    }

    // Step J (mod kPeriod): x_p, x_s1, x_s2 = level 0 at p, p - s1, p - 2 s1.
    // out[k] = level-M node k at p.
    template <int J>
    __device__ __forceinline__ void step(const Omega27 &om, float2 x_p, float2 x_s1, float2 x_s2,
                                         float2 (&out)[kN]) {
        if constexpr (M == 0) {
            out[0] = x_p;
        } else {
            bfly3(x_s2, x_s1, x_p, om.h, out[0], out[1], out[2]);
            level<J, 2>(om, out);
        }
    }

  private:
    template <int J, int T>
    __device__ __forceinline__ void level(const Omega27 &om, float2 (&cur)[kN]) {
        if constexpr (T <= M) {
            constexpr int s = pow3(M - T);
            constexpr int D = 2 * s;
            constexpr int H = pow3(T - 1);
            constexpr int off = fifo_off(T);
            constexpr int now = (J % D) * H;       // holds level T-1 from 2 s steps back
            constexpr int back1 = ((J + s) % D) * H;  // holds level T-1 from s steps back
            constexpr int tw = kMaxN3 / pow3(T);   // w_{3^T}^{-k} = w_27^{-k * tw}
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const float2 a2 = cur[i];
                const float2 a1 = fifo[off + back1 + i];
                const float2 a0 = fifo[off + now + i];
                fifo[off + now + i] = a2;
                const float2 b1 = i == 0 ? a1 : c_mul(om.w[(i * tw) % kMaxN3], a1);
                const float2 b2 = i == 0 ? a2 : c_mul(om.w[(2 * i * tw) % kMaxN3], a2);
                bfly3(a0, b1, b2, om.h, cur[i], cur[i + H], cur[i + 2 * H]);
            }
            level<J, T + 1>(om, cur);
        }
    }
};

}  // namespace swdft
