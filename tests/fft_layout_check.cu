// Host-side check of the team FFT's shared-memory layout and thread maps (team_fft.cuh),
// for every tile: test infrastructure, compiled and run by tests/test_fft_layout.py.
//
// For each geometry it checks, with the header's own map functions:
//   1. exchange 1: the words pass-1 threads write are distinct, inside the buffer (EXW),
//      and are exactly the words pass-2 threads read, each pass-2 thread finding the value
//      (row t1 = BY*ay + by + S*bx, column k1) its decomposition asks for;
//   2. exchange 2: every word a pass-3 thread reads was written (in the word it read in
//      exchange 1) by a pass-2 thread of the same warp, and the pass-3 reads cover every
//      value once;
//   3. banks: every warp instruction of passes 1, 2 and 3 touches 16 distinct 8-byte bank
//      pairs in each half-warp;
//   4. frequencies: (freq_ky, freq_kx) over the pass-3 layout cover the S x S spectrum once
//      and freq_place inverts them.
// Prints one line per geometry and exits with the number of failed checks.
#include <cstdio>
#include <vector>

#include "team_fft.cuh"

using namespace ptylm;

template <int LS, int LE>
int check_geometry() {
    using G = Geo<LS, LE>;
    int bad = 0;
    // 1. exchange 1
    std::vector<int> value(G::EXW, -1);   // which (t1, k) a word holds after the pass-1 stores
    for (int t1 = 0; t1 < G::T; ++t1)
        for (int k = 0; k < G::E; ++k) {
            const int w = p1_base<G>(t1) + k;
            if (w < 0 || w >= G::EXW || value[w] != -1) ++bad;
            else value[w] = t1 * G::E + k;
        }
    std::vector<int> reader(G::EXW, -1);  // the pass-2 thread that reads (and later writes) a word
    for (int t2 = 0; t2 < G::T; ++t2) {
        const int k1x = p2_k1x<G>(t2), by = p2_by<G>(t2);
        for (int ay = 0; ay < G::AY; ++ay)
            for (int bx = 0; bx < G::BX; ++bx) {
                const int w = ex_word<G>(by, ay, bx, k1x);
                const int t1 = G::BY * ay + by + G::S * bx;
                if (w < 0 || w >= G::EXW || value[w] != t1 * G::E + k1x || reader[w] != -1) ++bad;
                else reader[w] = t2;
            }
    }
    // 2. exchange 2
    if (G::BY > 1) {
        std::vector<int> seen(G::EXW, 0);
        for (int t3 = 0; t3 < G::T; ++t3) {
            const int k1x = p3_k1x<G>(t3), k2x = p3_k2x<G>(t3), k1y0 = p3_k1y0<G>(t3);
            for (int j = 0; j < G::G3; ++j)
                for (int by = 0; by < G::BY; ++by) {
                    const int w = ex_word<G>(by, k1y0 + G::BX * j, k2x, k1x);
                    if (w < 0 || w >= G::EXW || reader[w] < 0 || (reader[w] >> 5) != (t3 >> 5)) ++bad;
                    else ++seen[w];
                }
        }
        int covered = 0;
        for (int w = 0; w < G::EXW; ++w) {
            if (seen[w] > 1) ++bad;
            covered += seen[w];
        }
        if (covered != G::M) ++bad;
    }
    // 3. banks: 16 distinct (word mod 16) per half-warp and instruction
    auto distinct16 = [](const int* w) {
        unsigned mask = 0;
        for (int i = 0; i < 16; ++i) mask |= 1u << (w[i] & 15);
        return mask == 0xffffu;
    };
    int words[32];
    for (int w0 = 0; w0 < G::T; w0 += 32) {
        const int lanes = G::T - w0 < 32 ? G::T - w0 : 32;
        auto check = [&] {
            for (int h = 0; h + 16 <= lanes; h += 16)
                if (!distinct16(words + h)) ++bad;
        };
        for (int k = 0; k < G::E; ++k) {
            for (int l = 0; l < lanes; ++l) words[l] = p1_base<G>(w0 + l) + k;
            check();
        }
        for (int ay = 0; ay < G::AY; ++ay)
            for (int bx = 0; bx < G::BX; ++bx) {
                for (int l = 0; l < lanes; ++l)
                    words[l] = ex_word<G>(p2_by<G>(w0 + l), ay, bx, p2_k1x<G>(w0 + l));
                check();
            }
        if (G::BY > 1)
            for (int j = 0; j < G::G3; ++j)
                for (int by = 0; by < G::BY; ++by) {
                    for (int l = 0; l < lanes; ++l) {
                        const int t3 = w0 + l;
                        words[l] = ex_word<G>(by, p3_k1y0<G>(t3) + G::BX * j, p3_k2x<G>(t3), p3_k1x<G>(t3));
                    }
                    check();
                }
    }
    // 4. frequencies
    std::vector<int> hit(G::M, 0);
    for (int t3 = 0; t3 < G::T; ++t3)
        for (int e = 0; e < G::E; ++e) {
            const int ky = freq_ky<G>(t3), kx = freq_kx<G>(t3, e);
            if (ky < 0 || ky >= G::S || kx < 0 || kx >= G::S) {
                ++bad;
                continue;
            }
            ++hit[ky * G::S + kx];
            int t = -1, ee = -1;
            freq_place<G>(ky, kx, t, ee);
            if (t != t3 || ee != e) ++bad;
        }
    for (int i = 0; i < G::M; ++i)
        if (hit[i] != 1) ++bad;
    std::printf("S=%d E=%d T=%d BY=%d strides %d %d %d words %d (%.3f of S*S): %d failed checks\n", G::S, G::E, G::T,
                G::BY, G::EX_A, G::EX_B, G::EX_C, G::EXW, (double)G::EXW / G::M, bad);
    return bad;
}

int main() {
    int bad = 0;
    bad += check_geometry<5, 5>();
    bad += check_geometry<5, 4>();
    bad += check_geometry<6, 5>();
    bad += check_geometry<6, 4>();
    bad += check_geometry<7, 5>();
    return bad == 0 ? 0 : 1;
}
