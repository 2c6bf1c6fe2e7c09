// Streaming ternary and mixed-radix sliding trees: windows of 3^b 2^a samples (b >= 1,
// at most 64) along one axis; 3, 9 and 27 are the ternary trees.
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
// With radix-2 levels after the radix-3 ones (n = 3^b 2^a) the same holds level by level:
// a radix-2 level reads its level-(t-1) FIFO s_t steps back, and the residue split carries
// through because N_(t-1) is a multiple of 3.
#pragma once

#include "swdft_internal.h"
#include "tree_core.cuh"

namespace swdft {

__host__ __device__ constexpr int pow3(int m) { return m <= 0 ? 1 : 3 * pow3(m - 1); }

// w_n^{-j}, j < n (FP64-evaluated, FP32-rounded) for the window length n of one axis, and
// h = sin(pi/3) from the same table (-Im w_n^{-n/3}), for the radix-3 butterfly.
struct OmegaN {
    float2 w[kMaxN];
    float h;
};

// Y0 = B0 + B1 + B2, Y1 = B0 + w3^-1 B1 + w3^-2 B2, Y2 = B0 + w3^-2 B1 + w3^-1 B2,
// w3^-1 = -1/2 - i h, w3^-2 = -1/2 + i h: with s = B1 + B2, d = B1 - B2 and t = B0 - s/2,
// Y1 = t - i h d and Y2 = t + i h d, each component one fused multiply-add.
__device__ __forceinline__ void bfly3(float2 b0, float2 b1, float2 b2, float h, float2 &y0, float2 &y1,
                                      float2 &y2) {
    const float2 s = c_add(b1, b2);
    const float2 d = c_sub(b1, b2);
    const float2 t = make_float2(fmaf(-0.5f, s.x, b0.x), fmaf(-0.5f, s.y, b0.y));
    y0 = c_add(b0, s);
    y1 = make_float2(fmaf(h, d.y, t.x), fmaf(-h, d.x, t.y));
    y2 = make_float2(fmaf(-h, d.y, t.x), fmaf(h, d.x, t.y));
}

// Window lengths n = 3^B3 2^A2 (B3 >= 1): B3 radix-3 levels first, then A2 radix-2 levels.
// Level t has N_t = r_1 .. r_t nodes and reads level t-1 at p, p - s_t (and p - 2 s_t for
// radix 3), s_t = n / N_t:
//
//     T_t(p)[i] = sum_{d < r_t} w_{N_t}^{-i d} T_(t-1)(p - (r_t - 1 - d) s_t)[i mod N_(t-1)]
//
// (the ternary recurrence above with the radix chosen per level; for radix 2 the paper's).
__host__ __device__ constexpr int mixed_n(int B3, int A2) { return pow3(B3) << A2; }

// The tree split over three threads by node residue mod 3 (B3 >= 1).  Level 1 (radix 3) gives
// thread c its node c; every later level's node i is computed from node i mod N_(t-1) of the
// level before, a multiple of 3 apart, so thread c keeps only the nodes == c (mod 3) of every
// level, with no exchange and no node evaluated twice.  At a radix-3 level it evaluates the
// N_(t-1)/3 butterflies of 3 on i' == c (mod 3); at a radix-2 level the N_(t-1)/3 butterflies of
// 2 (nodes i' and i' + N_(t-1)).  Thread c produces the outputs k = c + 3 u, u < n/3.
template <int B3, int A2>
struct SlidingTreeMixed {
    static_assert(B3 >= 1 && B3 <= kMaxLog3 && A2 >= 0 && mixed_n(B3, A2) <= kMaxN,
                  "split trees: windows of 3^b 2^a <= 64 samples with b >= 1");
    static constexpr int L = B3 + A2;
    static constexpr int kN = mixed_n(B3, A2);
    static constexpr int kOut = kN / 3;  // outputs per thread
    static constexpr int kS1 = kN / 3;   // s_1: level 1 reads p, p - s_1, p - 2 s_1
    static constexpr int rad(int t) { return t <= B3 ? 3 : 2; }
    static constexpr int Nt(int t) { return t <= B3 ? pow3(t) : (pow3(B3) << (t - B3)); }
    static constexpr int st(int t) { return kN / Nt(t); }
    static constexpr int held(int t) { return t <= 1 ? 1 : Nt(t) / 3; }  // level-t nodes held
    // FIFO of level t-1 that level t reads: (r_t - 1) s_t slots of held(t-1) values
    static constexpr int depth(int t) { return (rad(t) - 1) * st(t); }
    static constexpr int kPeriod = L >= 2 ? depth(2) : 1;  // every depth divides it
    static constexpr int fifo_off(int t) {
        int o = 0;
        for (int u = 2; u < t; ++u) o += depth(u) * held(u - 1);
        return o;
    }
    static constexpr int kFifo = L >= 2 ? fifo_off(L + 1) : 0;
    // twiddles: level 1: w_3^{-c}, w_3^{-2c}; level t >= 2: w_{N_t}^{-i' d}, d = 1 .. r_t - 1,
    // for each i' = c + 3 a, a < held(t-1)
    static constexpr int tw_off(int t) {
        int o = 2;
        for (int u = 2; u < t; ++u) o += (rad(u) - 1) * held(u - 1);
        return o;
    }
    static constexpr int kTw = tw_off(L + 1);
    static constexpr bool depths_divide_period() {
        for (int t = 2; t <= L; ++t)
            if (kPeriod % depth(t) != 0) return false;
        return true;
    }
    static_assert(depths_divide_period(), "FIFO depths must divide the unroll period");

    float2 fifo[kFifo > 0 ? kFifo : 1];
    float2 tw[kTw];

    // scale: a factor applied to every output, folded into level 1 (its twiddles, and one
    // FMA for the untwiddled term); the levels after it are linear.  1 leaves the tree's
    // arithmetic as it is (fmaf(1, a, b) is a + b).
    __device__ __forceinline__ void init(int c, const OmegaN &om, float scale = 1.f) {
        tw[0] = c_scale(scale, om.w[(c * kS1) % kN]);
        tw[1] = c_scale(scale, om.w[(2 * c * kS1) % kN]);
        static_for<2, L + 1>([&](auto TT) {
            constexpr int t = decltype(TT)::value;
            static_for<0, held(t - 1)>([&](auto AA) {
                constexpr int a = decltype(AA)::value;
                const int ip = c + 3 * a;
                static_for<1, rad(t)>([&](auto DD) {
                    constexpr int d = decltype(DD)::value;
                    tw[tw_off(t) + (rad(t) - 1) * a + d - 1] = om.w[(ip * d * st(t)) % kN];
                });
            });
        });
#pragma unroll
        for (int i = 0; i < (kFifo > 0 ? kFifo : 1); ++i) fifo[i] = make_float2(0.f, 0.f);
    }

    // out[u] = level-L node c + 3 u at p, times the scale given to init (the same scale here);
    // x_p, x_s1, x_s2 = the data at p, p - s_1, p - 2 s_1.
    template <int J>
    __device__ __forceinline__ void step(float h, float scale, float2 x_p, float2 x_s1, float2 x_s2,
                                         float2 (&out)[kOut]) {
        // level 1, node c: x(p - 2 s1) + w_3^{-c} x(p - s1) + w_3^{-2c} x(p), scaled
        float2 cur[kOut];
        const float2 y = c_add(c_mul(tw[0], x_s1), c_mul(tw[1], x_p));
        cur[0] = make_float2(fmaf(scale, x_s2.x, y.x), fmaf(scale, x_s2.y, y.y));
        level<J, 2>(h, cur);
#pragma unroll
        for (int u = 0; u < kOut; ++u) out[u] = cur[u];
    }

  private:
    // cur holds level T-1's nodes c + 3 a (a < held(T-1)) in slots a; on return level T's
    // nodes c + 3 a' (a' < held(T)) in slots a'.
    template <int J, int T>
    __device__ __forceinline__ void level(float h, float2 (&cur)[kOut]) {
        if constexpr (T <= L) {
            constexpr int s = st(T);
            constexpr int D = depth(T);
            constexpr int HP = held(T - 1);  // level T-1 nodes held = butterflies here
            constexpr int off = fifo_off(T);
            constexpr int now = (J % D) * HP;
            constexpr int tb = tw_off(T);
            float2 nxt[kOut];
            if constexpr (rad(T) == 3) {
                constexpr int back1 = ((J + s) % D) * HP;
#pragma unroll
                for (int a = 0; a < HP; ++a) {
                    // node i' = c + 3 a of level T-1 at p (a2), p - s (a1), p - 2 s (a0)
                    const float2 a2 = cur[a];
                    const float2 a1 = fifo[off + back1 + a];
                    const float2 a0 = fifo[off + now + a];
                    fifo[off + now + a] = a2;
                    const float2 b1 = c_mul(tw[tb + 2 * a], a1);
                    const float2 b2 = c_mul(tw[tb + 2 * a + 1], a2);
                    // outputs i' + k N_(T-1) = c + 3 (a + k HP): slots a + k HP
                    bfly3(a0, b1, b2, h, nxt[a], nxt[a + HP], nxt[a + 2 * HP]);
                }
            } else {
#pragma unroll
                for (int a = 0; a < HP; ++a) {
                    // node i' = c + 3 a at p (a1) and p - s (a0): outputs i' and i' + N_(T-1)
                    const float2 a1 = cur[a];
                    const float2 a0 = fifo[off + now + a];
                    fifo[off + now + a] = a1;
                    const float2 b = c_mul(tw[tb + a], a1);
                    nxt[a] = c_add(a0, b);
                    nxt[a + HP] = c_sub(a0, b);
                }
            }
#pragma unroll
            for (int a = 0; a < rad(T) * HP; ++a) cur[a] = nxt[a];
            level<J, T + 1>(h, cur);
        }
    }
};

}  // namespace swdft
