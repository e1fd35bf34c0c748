// Host entry to the CRT reconstruction's rounding (bigfloat.cuh): the
// magnitude words of Z (little endian, 8 words), its sign and the scale s
// give hi + lo, the dd nearest to Z 2^s.  Built as a shared library for the
// CPU test.
#include <cstdint>

#include "bigfloat.cuh"

extern "C" void words_to_dd(const uint32_t *z, uint32_t neg, int s, double *out) {
    uint32_t w[8];
    for (int t = 0; t < 8; ++t) w[t] = z[t];
    mpdd::bigf::to_dd(mpdd::bigf::from_words<8>(w, neg, s), out[0], out[1]);
}
