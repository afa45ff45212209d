// team_fft.cuh -- register/shared-memory 2D FFT for one S x S patch per thread team.
//
// The far-field propagator of the model (Sec. 2, Eq. expected_count) is an S x S 2D DFT
// applied independently at every scan position.  A "team" of T = S*S/E threads owns one
// patch; every thread holds E complex values in registers (E = 32, or E = 16 for 32^2 and
// 64^2 patches, chosen per context or per batch schedule) and the 2D transform runs as
// three register passes separated by two shared-memory exchanges.  The first
// transformed dimension (d1) is the patch row index y, the second (d2) the column index x:
//
//   d1 = BX*a1 + b1  (E x BX = S)            d2 = BY*ay + by  (AY x BY = S, AY = E/BX)
//   pass 1   DFT_E over a1           -> k1, twiddle W_S^(b1*k1)     thread t1 = d2 + S*b1
//   pass 2   DFT_BX over b1 -> k2;  DFT_AY over ay -> k1y,
//            twiddle W_S^(by*k1y)                                  thread t2 = by + BY*k1
//   pass 3   DFT_BY over by          -> k2y      thread t3 = (k2, k1y0, k1), BY = BX^2 threads
//            per k1, for the G3 = E/BY values k1y = k1y0 + BX*j, j < G3
//   frequency index (k_d1, k_d2) = (k1 + E*k2, k1y + AY*k2y)
//
// Exchange 2 only moves data between the threads that share k1: BY pass-2 threads and BY
// pass-3 threads, which the maps above place in one warp (32/BY values of k1 per warp).
// Each pass-2 thread writes its exchange-2 values into the very slots it read in exchange 1,
// so exchange 2 needs no team barrier, only a warp barrier: a position's round trip
// (forward, spectral stage, inverse) passes two team barriers, both at exchange 1, and the
// warps run the rest of it without waiting for one another.
//
// In pass 1 the 32 lanes of a warp hold 32 consecutive columns of one row, so the patch
// gather and the scatter-add touch 256 contiguous bytes per warp instruction.
//
// The inverse runs the same passes backwards with conjugate twiddles, so a forward
// transform, an elementwise frequency-domain stage and an inverse transform need four
// exchanges and no transposition back to natural order: the frequency stage sees its
// elements in the "pass-3" layout and computes their frequency index instead.
//
// Exchange layout (units of 8-byte complex words), shared by both exchanges: a padded
// array word(by, ay, bx, k) = A*by + B*ay + C*bx + k for pass-1 row t1 = BY*ay + by + S*bx
// and k < E; exchange 2 puts the value (k2, k1y, by, k1) at word(by, k1y, k2, k1), the word
// its pass-2 thread read the input (ay = k1y, bx = k2) from.  Every access is a per-thread
// base plus a compile-time offset.  A 64-bit access is served per half-warp, so the strides'
// residues mod 16 are chosen to give each half-warp's 16 words distinct bank pairs in all
// three patterns: pass 1 (lanes vary t1's low bits), pass 2 (lanes vary by and k1's low
// bits) and pass 3 (lanes vary k2, k1y0 and k1's low bits):
//   BY = 16: A, B, C = 1, 1, 4 (mod 16);  BY = 4: A, B, C = 4, 1, 8, with the pass-3
//   half-warps taking the k1 of one parity;  BY = 1: B odd.
// The padding costs 3 % (S = 128) to 26 % (S = 32, E = 16) of the unpadded S*S words.
//
// Unnormalised transforms: forward then inverse multiplies by S*S; callers fold the
// orthonormal 1/S factors into their frequency-domain stage.
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace ptylm {

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
    return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// conj(a) * w
__device__ __forceinline__ float2 cconjmul(float2 a, float2 w) {
    return make_float2(a.x * w.x + a.y * w.y, a.x * w.y - a.y * w.x);
}

// cos(2 pi i / 32) for i = 0..8 (first octant), rounded to float.
__host__ __device__ constexpr float cos32_octant(int i) {
    return i == 0 ? 1.0f
         : i == 1 ? 9.807852507e-01f
         : i == 2 ? 9.238795042e-01f
         : i == 3 ? 8.314695954e-01f
         : i == 4 ? 7.071067691e-01f
         : i == 5 ? 5.555702448e-01f
         : i == 6 ? 3.826834261e-01f
         : i == 7 ? 1.950903237e-01f
         : 0.0f;
}
// cos(2 pi j / 32) for any integer j, by the symmetries of the cosine.
__host__ __device__ constexpr float cos32(int j) {
    j &= 31;
    return j <= 8 ? cos32_octant(j)
         : j <= 16 ? -cos32_octant(16 - j)
         : j <= 24 ? -cos32_octant(j - 16)
         : cos32_octant(32 - j);
}
// sin(x) = cos(x - pi/2)
__host__ __device__ constexpr float sin32(int j) { return cos32((j - 8) & 31); }

// a * W_32^J  with W = exp(-2 pi i / 32) (forward) or its conjugate (INV).
template <int J, bool INV>
__device__ __forceinline__ float2 twmul32(float2 a) {
    constexpr int j = J & 31;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 8) {
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (j == 16) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (j == 24) {
        return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else {
        constexpr float c = cos32(j);
        constexpr float s = INV ? sin32(j) : -sin32(j);
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

// In-register R-point DFT (R a power of two <= 32), natural order in and out, radix-2
// decimation in time.  After inlining, every index and twiddle is a compile-time constant.
template <int R, bool INV>
struct RegDFT;

template <bool INV>
struct RegDFT<1, INV> {
    __device__ __forceinline__ static void run(float2*) {}
};

template <bool INV>
struct RegDFT<2, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
};

// X = e + w o, Y = e - w o for w = W_32^J (conjugated when INV).  Trivial twiddles cost
// only the two complex additions.  A general twiddle w = c + i s is applied in the
// factored form w o = c (o + i (s/c) o) when |c| >= |s| (else s ((c/s) o + i o)), which
// folds the scaling into the additions: 6 FP32 instructions per butterfly instead of 8.
template <int J, bool INV>
__device__ __forceinline__ void twiddle_butterfly(float2 e, float2 o, float2& X, float2& Y) {
    constexpr int j = J & 31;
    if constexpr (j == 0 || j == 8 || j == 16 || j == 24) {
        const float2 t = twmul32<J, INV>(o);
        X = e + t;
        Y = e - t;
    } else {
        constexpr float c = cos32(j);
        constexpr float s = INV ? sin32(j) : -sin32(j);
        if constexpr ((c >= 0 ? c : -c) >= (s >= 0 ? s : -s)) {
            constexpr float r = s / c;  // w o = c (o.x - r o.y, o.y + r o.x)
            const float ux = fmaf(-r, o.y, o.x), uy = fmaf(r, o.x, o.y);
            X = make_float2(fmaf(c, ux, e.x), fmaf(c, uy, e.y));
            Y = make_float2(fmaf(-c, ux, e.x), fmaf(-c, uy, e.y));
        } else {
            constexpr float r = c / s;  // w o = s (r o.x - o.y, o.x + r o.y)
            const float ux = fmaf(r, o.x, -o.y), uy = fmaf(r, o.y, o.x);
            X = make_float2(fmaf(s, ux, e.x), fmaf(s, uy, e.y));
            Y = make_float2(fmaf(-s, ux, e.x), fmaf(-s, uy, e.y));
        }
    }
}

template <int K, int R, bool INV>
__device__ __forceinline__ void dit_butterfly(float2* v, const float2* e, const float2* o) {
    twiddle_butterfly<K * (32 / R), INV>(e[K], o[K], v[K], v[K + R / 2]);
}

template <int R, bool INV, int... Ks>
__device__ __forceinline__ void dit_combine(float2* v, const float2* e, const float2* o,
                                            std::integer_sequence<int, Ks...>) {
    (dit_butterfly<Ks, R, INV>(v, e, o), ...);
}

template <int R, bool INV>
struct RegDFT {
    static_assert(R >= 4 && R <= 32 && (R & (R - 1)) == 0, "radix must be a power of two <= 32");
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        RegDFT<R / 2, INV>::run(e);
        RegDFT<R / 2, INV>::run(o);
        dit_combine<R, INV>(v, e, o, std::make_integer_sequence<int, R / 2>{});
    }
};

// DFT of length R over v[base + STRIDE*i], i = 0..R-1 (base compile-time after unrolling).
template <int R, int STRIDE, bool INV>
__device__ __forceinline__ void dft_strided(float2* v, int base) {
    if constexpr (R > 1) {
        float2 t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[base + STRIDE * i];
        RegDFT<R, INV>::run(t);
#pragma unroll
        for (int i = 0; i < R; ++i) v[base + STRIDE * i] = t[i];
    }
}

// smallest integer >= x congruent to r mod 16
__host__ __device__ constexpr int ex_up16(int x, int r) { return x + (((r - x) % 16) + 16) % 16; }

// Geometry of the three-pass decomposition for S = 2^LS with E = 2^LE values per thread.
template <int LS, int LE = 5>
struct Geo {
    static_assert(LS >= 5 && LS <= 7, "supported patch sides: 32, 64, 128");
    static_assert(LE == 5 || (LE == 4 && LS <= 6), "values per thread: 32, or 16 for sides 32 and 64");
    static constexpr int LOG_S = LS;
    static constexpr int LOG_E = LE;
    static constexpr int S = 1 << LS;
    static constexpr int M = S * S;
    static constexpr int E = 1 << LE;    // complex values per thread
    static constexpr int T = M / E;      // threads per team
    static constexpr int BX = S / E;
    static constexpr int AY = E / BX;
    static constexpr int BY = S / AY;
    static constexpr int G3 = E / BY;    // pass-3 groups per thread
    static constexpr int LOG_BX = LS - LE;
    static constexpr int LOG_BY = 2 * LOG_BX;
    static_assert(BY <= E, "pass 3 must fit one thread's values");
    static_assert(BY == BX * BX && (BY == 1 || BY == 4 || BY == 16), "pass-3 thread map");
    // exchange strides (see the layout above) and the words one team's buffer takes
    static constexpr int EX_A = BY == 16 ? ex_up16(E, 1) : BY == 4 ? ex_up16(E, 4) : E;
    static constexpr int EX_B = ex_up16((BY - 1) * EX_A + E, 1);
    static constexpr int EX_C = BX > 1 ? ex_up16((AY - 1) * EX_B + (BY - 1) * EX_A + E, BY == 16 ? 4 : 8) : AY * EX_B;
    // (rounded up to an even count, so that every team's buffer starts 16-byte aligned)
    static constexpr int EXW = ((BX - 1) * EX_C + (AY - 1) * EX_B + (BY - 1) * EX_A + E + 1) & ~1;
    static_assert(EXW >= M, "exchange buffer");
    static constexpr int TW_WORDS = 2 * S;   // shared-memory twiddles (fill_twiddles)
    // teams per CTA of the single-problem kernels: several only for one-warp teams, whose
    // barriers are warp-local (teams in one CTA may run different numbers of positions)
    static constexpr int TEAMS = (T > 32) ? 1 : 128 / T;
    static constexpr int THREADS = T * TEAMS;
};

// Twiddles in shared memory, TW_WORDS = 2S entries per tile: tw[j] = W_S^j (j < S) and
// tw[S + BY*k1y + by] = W_S^(by*k1y), pass 2's twiddles laid out so that its lanes (which
// vary by) read consecutive words.  Filled from the S-entry table w_s by threads
// i0, i0 + step, ...
template <class G>
__device__ __forceinline__ void fill_twiddles(float2* tw, const float2* w_s, int i0, int step) {
    for (int i = i0; i < G::S; i += step) {
        tw[i] = w_s[i];
        tw[G::S + i] = w_s[(i % G::BY) * (i / G::BY)];
    }
}

template <class G>
__device__ __forceinline__ void team_sync() {
    if constexpr (G::T == 32) __syncwarp();
    else __syncthreads();
}

// ---- pass 1: thread t1 = d2 + S*b1 holds v[a1] = element (d1 = BX*a1 + b1, d2) ----------
// Compiler scheduling fence: keeps loads from being hoisted across it, which bounds the
// registers held by loads in flight (the 32 data values already take 64 registers).
__device__ __forceinline__ void sched_fence() { asm volatile("" ::: "memory"); }

template <class G>
__device__ __forceinline__ void pass1_fwd(float2* v, const float2* tw, int t1) {
    RegDFT<G::E, false>::run(v);
    if constexpr (G::BX > 1) {
        const int bx = (t1 >> G::LOG_S) & (G::BX - 1);
#pragma unroll
        for (int k0 = 0; k0 < G::E; k0 += 8) {
            float2 w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = tw[bx * (k0 + i)];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (k0 + i > 0) v[k0 + i] = cmul(v[k0 + i], w[i]);
            sched_fence();
        }
    }
}

template <class G>
__device__ __forceinline__ void pass1_inv(float2* v) {
    RegDFT<G::E, true>::run(v);
}

// ---- exchange layout and thread maps -------------------------------------------------
template <class G>
__host__ __device__ __forceinline__ int ex_word(int by, int ay, int bx, int k) {
    return G::EX_A * by + G::EX_B * ay + G::EX_C * bx + k;
}
// pass-1 row t1 = BY*ay + by + S*bx;  pass-2 thread t2 = by + BY*k1x;  pass-3 thread
// t3 = k2x + BX*k1y0 + BY*k1x (BY = 16, 1) or, for BY = 4, k2x + 2*k1y0 + 4*m + 16*h + 32*w
// with k1x = 8w + 2m + h.  t < T = E*BY: the masks state the ranges.
template <class G>
__host__ __device__ __forceinline__ int p1_base(int t1) {
    return ex_word<G>(t1 & (G::BY - 1), (t1 >> G::LOG_BY) & (G::AY - 1), (t1 >> G::LOG_S) & (G::BX - 1), 0);
}
template <class G>
__host__ __device__ __forceinline__ int p2_k1x(int t2) { return (t2 >> G::LOG_BY) & (G::E - 1); }
template <class G>
__host__ __device__ __forceinline__ int p2_by(int t2) { return t2 & (G::BY - 1); }
template <class G>
__host__ __device__ __forceinline__ int p3_k1x(int t3) {
    if constexpr (G::BY == 4) return (((t3 >> 5) << 3) | (((t3 >> 2) & 3) << 1) | ((t3 >> 4) & 1)) & (G::E - 1);
    else return (t3 >> G::LOG_BY) & (G::E - 1);
}
template <class G>
__host__ __device__ __forceinline__ int p3_k2x(int t3) { return t3 & (G::BX - 1); }
template <class G>
__host__ __device__ __forceinline__ int p3_k1y0(int t3) { return (t3 >> G::LOG_BX) & (G::BX - 1); }

// ---- exchange 1 --------------------------------------------------------------------
template <class G>
__device__ __forceinline__ void ex1_store_from_p1(float2* sm, const float2* v, int t1) {
    float2* row = sm + p1_base<G>(t1);
#pragma unroll
    for (int k = 0; k < G::E; ++k) row[k] = v[k];
}
template <class G>
__device__ __forceinline__ void ex1_load_to_p1(const float2* sm, float2* v, int t1) {
    const float2* row = sm + p1_base<G>(t1);
#pragma unroll
    for (int k = 0; k < G::E; ++k) v[k] = row[k];
}
// pass-2 register layout: v[ay*BX + bx] (before pass 2) / v[k1y*BX + k2x] (after)
template <class G>
__device__ __forceinline__ const float2* p2_words(const float2* sm, int t2) {
    return sm + ex_word<G>(p2_by<G>(t2), 0, 0, p2_k1x<G>(t2));
}
template <class G>
__device__ __forceinline__ void ex1_load_to_p2(const float2* sm, float2* v, int t2) {
    const float2* q = p2_words<G>(sm, t2);
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay)
#pragma unroll
        for (int bx = 0; bx < G::BX; ++bx) v[ay * G::BX + bx] = q[G::EX_B * ay + G::EX_C * bx];
}
template <class G>
__device__ __forceinline__ void ex1_store_from_p2(float2* sm, const float2* v, int t2) {
    float2* q = const_cast<float2*>(p2_words<G>(sm, t2));
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay)
#pragma unroll
        for (int bx = 0; bx < G::BX; ++bx) q[G::EX_B * ay + G::EX_C * bx] = v[ay * G::BX + bx];
}

// ---- pass 2 ----------------------------------------------------------------------------
template <class G>
__device__ __forceinline__ void pass2_fwd(float2* v, const float2* tw, int t2) {
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay) dft_strided<G::BX, 1, false>(v, ay * G::BX);
#pragma unroll
    for (int k2x = 0; k2x < G::BX; ++k2x) dft_strided<G::AY, G::BX, false>(v, k2x);
    if constexpr (G::BY > 1) {
        const int by = p2_by<G>(t2);
#pragma unroll
        for (int k1y = 1; k1y < G::AY; ++k1y) {
            const float2 w = tw[G::S + G::BY * k1y + by];   // W_S^(by*k1y), lanes vary by
#pragma unroll
            for (int k2x = 0; k2x < G::BX; ++k2x) v[k1y * G::BX + k2x] = cmul(v[k1y * G::BX + k2x], w);
        }
    }
}

template <class G>
__device__ __forceinline__ void pass2_inv(float2* v, const float2* tw, int t2) {
    const int k1x = p2_k1x<G>(t2);
    if constexpr (G::BY > 1) {
        const int by = p2_by<G>(t2);
#pragma unroll
        for (int k1y = 1; k1y < G::AY; ++k1y) {
            const float2 w = tw[G::S + G::BY * k1y + by];   // W_S^(by*k1y), lanes vary by
#pragma unroll
            for (int k2x = 0; k2x < G::BX; ++k2x) v[k1y * G::BX + k2x] = cmulc(v[k1y * G::BX + k2x], w);
        }
    }
#pragma unroll
    for (int k2x = 0; k2x < G::BX; ++k2x) dft_strided<G::AY, G::BX, true>(v, k2x);
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay) dft_strided<G::BX, 1, true>(v, ay * G::BX);
    if constexpr (G::BX > 1) {
#pragma unroll
        for (int bx = 1; bx < G::BX; ++bx) {
            const float2 w = tw[bx * k1x];
#pragma unroll
            for (int ay = 0; ay < G::AY; ++ay) v[ay * G::BX + bx] = cmulc(v[ay * G::BX + bx], w);
        }
    }
}

// ---- exchange 2 (skipped when BY == 1: the data already sits in the right thread) -----
// Value (k2x, k1y, by, k1x) sits in the word pass-2 thread (by, k1x) read its input
// (ay = k1y, bx = k2x) from in exchange 1.
template <class G>
__device__ __forceinline__ void ex2_store_from_p2(float2* sm, const float2* v, int t2) {
    ex1_store_from_p2<G>(sm, v, t2);   // same words, the pass-2 output in the input's place
}
template <class G>
__device__ __forceinline__ void ex2_load_to_p2(const float2* sm, float2* v, int t2) {
    ex1_load_to_p2<G>(sm, v, t2);
}
// pass-3 register layout: v[j*BY + by] (before pass 3) / v[j*BY + k2y] (after); the words
// of group j start at p3_words(sm, t3) + EX_B*BX*j, one every EX_A
template <class G, class W>
__device__ __forceinline__ W* p3_words(W* sm, int t3) {
    return sm + ex_word<G>(0, p3_k1y0<G>(t3), p3_k2x<G>(t3), p3_k1x<G>(t3));
}
template <class G>
__device__ __forceinline__ void ex2_load_to_p3(const float2* sm, float2* v, int t3) {
    const float2* q = p3_words<G>(sm, t3);
#pragma unroll
    for (int j = 0; j < G::G3; ++j)
#pragma unroll
        for (int by = 0; by < G::BY; ++by) v[j * G::BY + by] = q[G::EX_B * G::BX * j + G::EX_A * by];
}
template <class G>
__device__ __forceinline__ void ex2_store_from_p3(float2* sm, const float2* v, int t3) {
    float2* q = p3_words<G>(sm, t3);
#pragma unroll
    for (int j = 0; j < G::G3; ++j)
#pragma unroll
        for (int by = 0; by < G::BY; ++by) q[G::EX_B * G::BX * j + G::EX_A * by] = v[j * G::BY + by];
}

// ---- pass 3 ----------------------------------------------------------------------------
template <class G>
__device__ __forceinline__ void pass3_fwd(float2* v) {
#pragma unroll
    for (int j = 0; j < G::G3; ++j) dft_strided<G::BY, 1, false>(v, j * G::BY);
}
template <class G>
__device__ __forceinline__ void pass3_inv(float2* v) {
#pragma unroll
    for (int j = 0; j < G::G3; ++j) dft_strided<G::BY, 1, true>(v, j * G::BY);
}

// Frequency index (row ky, column kx) of register element e in the pass-3 layout of
// thread t3: the row frequency comes from the first transformed dimension.
template <class G>
__host__ __device__ __forceinline__ int freq_ky(int t3) { return p3_k1x<G>(t3) + G::E * p3_k2x<G>(t3); }
template <class G>
__host__ __device__ __forceinline__ int freq_kx(int t3, int e) {
    const int j = e / G::BY, k2y = e % G::BY;
    return p3_k1y0<G>(t3) + G::BX * j + G::AY * k2y;
}
// The inverse: thread t3 and element e of the pass-3 layout that hold frequency (ky, kx).
template <class G>
__host__ __device__ __forceinline__ void freq_place(int ky, int kx, int& t3, int& e) {
    const int k1x = ky & (G::E - 1), k2x = ky >> G::LOG_E;
    const int k1y = kx % G::AY, k2y = kx / G::AY, k1y0 = k1y % G::BX, j = k1y / G::BX;
    e = j * G::BY + k2y;
    if constexpr (G::BY == 4) t3 = k2x + 2 * k1y0 + 4 * ((k1x >> 1) & 3) + 16 * (k1x & 1) + 32 * (k1x >> 3);
    else t3 = k2x + G::BX * k1y0 + G::BY * k1x;
}

// ---- whole transforms ------------------------------------------------------------------
// Forward: v in pass-1 layout (natural spatial data)  ->  v in pass-3 layout (spectrum).
template <class G>
__device__ __forceinline__ void team_fft_fwd(float2* v, float2* sm, const float2* tw, int tid) {
    pass1_fwd<G>(v, tw, tid);
    ex1_store_from_p1<G>(sm, v, tid);
    team_sync<G>();
    ex1_load_to_p2<G>(sm, v, tid);
    pass2_fwd<G>(v, tw, tid);
    if constexpr (G::BY > 1) {
        ex2_store_from_p2<G>(sm, v, tid);  // into the slots this thread has just read
        __syncwarp();
        ex2_load_to_p3<G>(sm, v, tid);
        pass3_fwd<G>(v);
    }
}

// Inverse: v in pass-3 layout (spectrum)  ->  v in pass-1 layout (spatial data).
// Its first shared-memory writes go to exactly the slots the same thread read last in
// team_fft_fwd, so it may follow team_fft_fwd without a barrier; after any other use of
// sm the caller synchronises the team first.  Exchange 2 stays within each warp, and the
// exchange-1 stores that follow it go to the slots the same thread has just read.
template <class G>
__device__ __forceinline__ void team_fft_inv(float2* v, float2* sm, const float2* tw, int tid) {
    if constexpr (G::BY > 1) {
        pass3_inv<G>(v);
        ex2_store_from_p3<G>(sm, v, tid);
        __syncwarp();
        ex2_load_to_p2<G>(sm, v, tid);
    }
    pass2_inv<G>(v, tw, tid);
    ex1_store_from_p2<G>(sm, v, tid);
    team_sync<G>();
    ex1_load_to_p1<G>(sm, v, tid);
    pass1_inv<G>(v);
}

// Forward transform, an elementwise spectral stage and the inverse transform in one go
// (v: pass-1 layout in and out).  Pass 3 runs one group of BY values at a time straight
// from / back to the thread's own exchange slots, so the spectral stage only holds one
// group (2*BY registers) plus whatever it loads: `stage(g, j)` receives the group's BY
// spectral values g[k2y] (element e = j*BY + k2y of the pass-3 layout) and overwrites them
// with the values to transform back.
template <class G, bool TEAM_PRE, class Stage, class Pre>
__device__ __forceinline__ void team_fft_roundtrip_impl(float2* v, float2* sm, const float2* tw, int tid,
                                                        Stage&& stage, Pre&& before_pass3);

template <class G, class Stage>
__device__ __forceinline__ void team_fft_roundtrip(float2* v, float2* sm, const float2* tw, int tid,
                                                   Stage&& stage) {
    team_fft_roundtrip_impl<G, false>(v, sm, tw, tid, stage, [] {});
}

// As above, with `before_pass3()` run by every thread just before pass 3 when BY > 1,
// followed by a team barrier (so data the spectral stage reads from shared memory, written
// asynchronously by the whole team, can be waited for there); when BY == 1 it runs before
// the first stage call with no barrier after it.  Without it (the overload above) exchange
// 2 and pass 3 need only warp barriers.
template <class G, class Stage, class Pre>
__device__ __forceinline__ void team_fft_roundtrip(float2* v, float2* sm, const float2* tw, int tid,
                                                   Stage&& stage, Pre&& before_pass3) {
    team_fft_roundtrip_impl<G, true>(v, sm, tw, tid, stage, before_pass3);
}

template <class G, bool TEAM_PRE, class Stage, class Pre>
__device__ __forceinline__ void team_fft_roundtrip_impl(float2* v, float2* sm, const float2* tw, int tid,
                                                        Stage&& stage, Pre&& before_pass3) {
    pass1_fwd<G>(v, tw, tid);
    ex1_store_from_p1<G>(sm, v, tid);
    team_sync<G>();
    ex1_load_to_p2<G>(sm, v, tid);
    pass2_fwd<G>(v, tw, tid);
    if constexpr (G::BY > 1) {
        ex2_store_from_p2<G>(sm, v, tid);  // into the slots this thread has just read
        before_pass3();
        if constexpr (TEAM_PRE) team_sync<G>();
        else __syncwarp();
        float2* q3 = p3_words<G>(sm, tid);
#pragma unroll 1
        for (int j = 0; j < G::G3; ++j) {
            float2 g[G::BY];
            float2* q = q3 + G::EX_B * G::BX * j;
#pragma unroll
            for (int by = 0; by < G::BY; ++by) g[by] = q[G::EX_A * by];
            RegDFT<G::BY, false>::run(g);
            stage(g, j);
            RegDFT<G::BY, true>::run(g);
#pragma unroll
            for (int by = 0; by < G::BY; ++by) q[G::EX_A * by] = g[by];
        }
        __syncwarp();
        ex2_load_to_p2<G>(sm, v, tid);   // the exchange-1 stores below go to these same slots
    } else {
        // BY == 1: the pass-2 registers already hold the spectrum, one value per group.
        before_pass3();
#pragma unroll
        for (int j = 0; j < G::G3; ++j) stage(v + j, j);
    }
    pass2_inv<G>(v, tw, tid);
    ex1_store_from_p2<G>(sm, v, tid);
    team_sync<G>();
    ex1_load_to_p1<G>(sm, v, tid);
    pass1_inv<G>(v);
}

}  // namespace ptylm
