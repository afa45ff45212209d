// team_fft.cuh -- register/shared-memory 2D FFT for one S x S patch per thread team.
//
// The far-field propagator of the model (Sec. 2, Eq. expected_count) is an S x S 2D DFT
// applied independently at every scan position.  A "team" of T = S*S/E threads owns one
// patch; every thread holds E complex values in registers (E = 32 everywhere except the
// batched kernels, which may run 32^2 and 64^2 patches with E = 16) and the 2D transform
// runs as three register passes separated by two shared-memory exchanges.  The first
// transformed dimension (d1) is the patch row index y, the second (d2) the column index x:
//
//   d1 = BX*a1 + b1  (E x BX = S)            d2 = BY*ay + by  (AY x BY = S, AY = E/BX)
//   pass 1   DFT_E over a1           -> k1, twiddle W_S^(b1*k1)     thread t1 = d2 + S*b1
//   pass 2   DFT_BX over b1 -> k2;  DFT_AY over ay -> k1y,
//            twiddle W_S^(by*k1y)                                  thread t2 = k1 + E*by
//   pass 3   DFT_BY over by          -> k2y                         thread (kd1, k1y)
//   frequency index (k_d1, k_d2) = (k1 + E*k2, k1y + AY*k2y)
//
// In pass 1 the 32 lanes of a warp hold 32 consecutive columns of one row, so the patch
// gather and the scatter-add touch 256 contiguous bytes per warp instruction.
//
// The inverse runs the same passes backwards with conjugate twiddles, so a forward
// transform, an elementwise frequency-domain stage and an inverse transform need four
// exchanges and no transposition back to natural order: the frequency stage sees its
// elements in the "pass-3" layout and computes their frequency index instead.
//
// Exchange layouts (units of 8-byte complex words):
//   ex1 (pass 1 <-> pass 2):  slot(t1, k1) = t1*E + (k1 ^ (t1 & (E-1)))
//        writers vary t1 across lanes, readers vary k1: the XOR swizzle keeps both
//        conflict-free (for E = 16 within each half-warp, the unit of a 64-bit access).
//   ex2 (pass 2 <-> pass 3):  slot = ((k2*AY + k1y)*BY + by)*E + k1
//        both sides have lanes = k1, so plain row-major is conflict-free.
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
    static_assert(BY <= E, "pass 3 must fit one thread's values");
    // teams per CTA of the single-problem kernels: several only for one-warp teams, whose
    // barriers are warp-local (teams in one CTA may run different numbers of positions)
    static constexpr int TEAMS = (T > 32) ? 1 : 128 / T;
    static constexpr int THREADS = T * TEAMS;
};

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

// ---- exchange 1 --------------------------------------------------------------------
template <class G>
__device__ __forceinline__ void ex1_store_from_p1(float2* sm, const float2* v, int t1) {
    const int sw = t1 & (G::E - 1);
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[t1 * G::E + (k ^ sw)] = v[k];
}
template <class G>
__device__ __forceinline__ void ex1_load_to_p1(const float2* sm, float2* v, int t1) {
    const int sw = t1 & (G::E - 1);
#pragma unroll
    for (int k = 0; k < G::E; ++k) v[k] = sm[t1 * G::E + (k ^ sw)];
}
// pass-2 register layout: v[ay*BX + bx] (before pass 2) / v[k1y*BX + k2x] (after)
template <class G>
__device__ __forceinline__ void ex1_load_to_p2(const float2* sm, float2* v, int t2) {
    const int k1x = t2 & (G::E - 1), by = (t2 >> G::LOG_E) & (G::BY - 1);  // t2 < T = E BY: the mask states the range
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay)
#pragma unroll
        for (int bx = 0; bx < G::BX; ++bx) {
            const int t1 = (G::BY * ay + by) + G::S * bx;
            v[ay * G::BX + bx] = sm[t1 * G::E + (k1x ^ (t1 & (G::E - 1)))];
        }
}
template <class G>
__device__ __forceinline__ void ex1_store_from_p2(float2* sm, const float2* v, int t2) {
    const int k1x = t2 & (G::E - 1), by = (t2 >> G::LOG_E) & (G::BY - 1);  // t2 < T = E BY: the mask states the range
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay)
#pragma unroll
        for (int bx = 0; bx < G::BX; ++bx) {
            const int t1 = (G::BY * ay + by) + G::S * bx;
            sm[t1 * G::E + (k1x ^ (t1 & (G::E - 1)))] = v[ay * G::BX + bx];
        }
}

// ---- pass 2 ----------------------------------------------------------------------------
template <class G>
__device__ __forceinline__ void pass2_fwd(float2* v, const float2* tw, int t2) {
#pragma unroll
    for (int ay = 0; ay < G::AY; ++ay) dft_strided<G::BX, 1, false>(v, ay * G::BX);
#pragma unroll
    for (int k2x = 0; k2x < G::BX; ++k2x) dft_strided<G::AY, G::BX, false>(v, k2x);
    if constexpr (G::BY > 1) {
        const int by = (t2 >> G::LOG_E) & (G::BY - 1);  // t2 < T = E BY: the mask states the range
#pragma unroll
        for (int k1y = 1; k1y < G::AY; ++k1y) {
            const float2 w = tw[by * k1y];
#pragma unroll
            for (int k2x = 0; k2x < G::BX; ++k2x) v[k1y * G::BX + k2x] = cmul(v[k1y * G::BX + k2x], w);
        }
    }
}

template <class G>
__device__ __forceinline__ void pass2_inv(float2* v, const float2* tw, int t2) {
    const int k1x = t2 & (G::E - 1);
    if constexpr (G::BY > 1) {
        const int by = (t2 >> G::LOG_E) & (G::BY - 1);  // t2 < T = E BY: the mask states the range
#pragma unroll
        for (int k1y = 1; k1y < G::AY; ++k1y) {
            const float2 w = tw[by * k1y];
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
template <class G>
__device__ __forceinline__ int ex2_slot(int k2x, int k1y, int by, int k1x) {
    return ((k2x * G::AY + k1y) * G::BY + by) * G::E + k1x;
}
template <class G>
__device__ __forceinline__ void ex2_store_from_p2(float2* sm, const float2* v, int t2) {
    const int k1x = t2 & (G::E - 1), by = (t2 >> G::LOG_E) & (G::BY - 1);  // t2 < T = E BY: the mask states the range
#pragma unroll
    for (int k1y = 0; k1y < G::AY; ++k1y)
#pragma unroll
        for (int k2x = 0; k2x < G::BX; ++k2x)
            sm[ex2_slot<G>(k2x, k1y, by, k1x)] = v[k1y * G::BX + k2x];
}
template <class G>
__device__ __forceinline__ void ex2_load_to_p2(const float2* sm, float2* v, int t2) {
    const int k1x = t2 & (G::E - 1), by = (t2 >> G::LOG_E) & (G::BY - 1);  // t2 < T = E BY: the mask states the range
#pragma unroll
    for (int k1y = 0; k1y < G::AY; ++k1y)
#pragma unroll
        for (int k2x = 0; k2x < G::BX; ++k2x)
            v[k1y * G::BX + k2x] = sm[ex2_slot<G>(k2x, k1y, by, k1x)];
}
// pass-3 register layout: v[j*BY + by] (before pass 3) / v[j*BY + k2y] (after)
template <class G>
__device__ __forceinline__ void ex2_load_to_p3(const float2* sm, float2* v, int t3) {
    const int k1x = t3 & (G::E - 1), k2x = (t3 & (G::S - 1)) >> G::LOG_E, k1y0 = t3 >> G::LOG_S;
#pragma unroll
    for (int j = 0; j < G::G3; ++j)
#pragma unroll
        for (int by = 0; by < G::BY; ++by)
            v[j * G::BY + by] = sm[ex2_slot<G>(k2x, k1y0 + G::BX * j, by, k1x)];
}
template <class G>
__device__ __forceinline__ void ex2_store_from_p3(float2* sm, const float2* v, int t3) {
    const int k1x = t3 & (G::E - 1), k2x = (t3 & (G::S - 1)) >> G::LOG_E, k1y0 = t3 >> G::LOG_S;
#pragma unroll
    for (int j = 0; j < G::G3; ++j)
#pragma unroll
        for (int by = 0; by < G::BY; ++by)
            sm[ex2_slot<G>(k2x, k1y0 + G::BX * j, by, k1x)] = v[j * G::BY + by];
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
__device__ __forceinline__ int freq_ky(int t3) { return t3 & (G::S - 1); }
template <class G>
__device__ __forceinline__ int freq_kx(int t3, int e) {
    const int j = e / G::BY, k2y = e % G::BY;
    return (t3 >> G::LOG_S) + G::BX * j + G::AY * k2y;
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
        team_sync<G>();  // all ex1 reads done before ex2 overwrites
        ex2_store_from_p2<G>(sm, v, tid);
        team_sync<G>();
        ex2_load_to_p3<G>(sm, v, tid);
        pass3_fwd<G>(v);
    }
}

// Inverse: v in pass-3 layout (spectrum)  ->  v in pass-1 layout (spatial data).
// Its first shared-memory writes go to exactly the slots the same thread read last in
// team_fft_fwd, so it may follow team_fft_fwd without a barrier; after any other use of
// sm the caller synchronises the team first.
template <class G>
__device__ __forceinline__ void team_fft_inv(float2* v, float2* sm, const float2* tw, int tid) {
    if constexpr (G::BY > 1) {
        pass3_inv<G>(v);
        ex2_store_from_p3<G>(sm, v, tid);
        team_sync<G>();
        ex2_load_to_p2<G>(sm, v, tid);
        team_sync<G>();  // all ex2 reads done before ex1 overwrites
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
template <class G, class Stage>
__device__ __forceinline__ void team_fft_roundtrip(float2* v, float2* sm, const float2* tw, int tid,
                                                   Stage&& stage) {
    team_fft_roundtrip<G>(v, sm, tw, tid, stage, [] {});
}

// As above, with `before_pass3()` run by every thread just before the barrier that precedes
// pass 3 when BY > 1 (so data the spectral stage reads from shared memory, written
// asynchronously, can be waited for there); when BY == 1 it runs before the first stage
// call with no barrier after it.
template <class G, class Stage, class Pre>
__device__ __forceinline__ void team_fft_roundtrip(float2* v, float2* sm, const float2* tw, int tid,
                                                   Stage&& stage, Pre&& before_pass3) {
    pass1_fwd<G>(v, tw, tid);
    ex1_store_from_p1<G>(sm, v, tid);
    team_sync<G>();
    ex1_load_to_p2<G>(sm, v, tid);
    pass2_fwd<G>(v, tw, tid);
    if constexpr (G::BY > 1) {
        team_sync<G>();  // all ex1 reads done before ex2 overwrites
        ex2_store_from_p2<G>(sm, v, tid);
        before_pass3();
        team_sync<G>();
        const int k1x = tid & (G::E - 1), k2x = (tid & (G::S - 1)) >> G::LOG_E, k1y0 = (tid >> G::LOG_S) & (G::BX - 1);
#pragma unroll 1
        for (int j = 0; j < G::G3; ++j) {
            float2 g[G::BY];
            const int base = ex2_slot<G>(k2x, k1y0 + G::BX * j, 0, k1x);
#pragma unroll
            for (int by = 0; by < G::BY; ++by) g[by] = sm[base + by * G::E];
            RegDFT<G::BY, false>::run(g);
            stage(g, j);
            RegDFT<G::BY, true>::run(g);
#pragma unroll
            for (int by = 0; by < G::BY; ++by) sm[base + by * G::E] = g[by];
        }
        team_sync<G>();
        ex2_load_to_p2<G>(sm, v, tid);
        team_sync<G>();  // all ex2 reads done before ex1 overwrites
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
