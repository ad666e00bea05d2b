// Host-side driver for the integer-only conversions of the FP32-phase path
// (fixed-point fractions, double->float, float->double).  Reads commands from stdin:
//   F r l      -> round(r / l * 2^32) mod 2^32 with 1/l taken as the double 1.0 / l
//   D x        -> bits of the nearest float to x
//   W fbits    -> bits of the double equal to the float with bits fbits
#include <cstdio>
#include <cstring>

#include "../../paper_2110_14362_gb300/csrc/rbe_device.cuh"

static rbe::FixScale scale_of(double ell)
{
    const double inv = 1.0 / ell;
    unsigned long long b;
    std::memcpy(&b, &inv, 8);
    const int e = (int)((b >> 52) & 0x7ff) - 1075;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return rbe::FixScale{mant << 11, e - 11};
}

int main()
{
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'F') {
            double r, l;
            if (std::scanf("%lf %lf", &r, &l) != 2) return 1;
            unsigned long long rb;
            std::memcpy(&rb, &r, 8);
            std::printf("%u\n", rbe::fixed_frac_int(rb, scale_of(l)));
        } else if (op == 'D') {
            double x;
            if (std::scanf("%lf", &x) != 1) return 1;
            unsigned long long xb;
            std::memcpy(&xb, &x, 8);
            const float f = rbe::double_to_float_int(xb);
            unsigned int fb;
            std::memcpy(&fb, &f, 4);
            std::printf("%u\n", fb);
        } else if (op == 'W') {
            unsigned int fb;
            if (std::scanf("%u", &fb) != 1) return 1;
            std::printf("%llu\n", rbe::float_to_double_bits(fb));
        }
    }
    return 0;
}
