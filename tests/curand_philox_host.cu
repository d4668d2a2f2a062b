// Host-side call of NVIDIA's Philox4x32-10 from the CUDA toolkit header
// curand_philox4x32_x.h (an implementation independent of the oracle's), used
// only by tests to pin the oracle's generator.  Reads "c0 c1 c2 c3 k0 k1"
// lines (hex) on stdin and prints the four output words per line.
#define QUALIFIERS static inline __host__ __device__
#include <cstdio>
#include <curand_philox4x32_x.h>

int main() {
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%x %x %x %x %x %x", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        uint4 c = make_uint4(c0, c1, c2, c3);
        uint2 k = make_uint2(k0, k1);
        uint4 o = curand_Philox4x32_10(c, k);
        std::printf("%08x %08x %08x %08x\n", o.x, o.y, o.z, o.w);
    }
    return 0;
}
