// philox.cuh -- Philox4x32-10 counter-based generator for device code.
//
// Written from the published definition (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): each of the ten
// rounds multiplies counter words 0 and 2 by two fixed odd constants
// (32x32 -> 64 bits), xors the high halves with the other two counter words
// and the key, and permutes the words; the key advances by the two Weyl
// constants between rounds.  One call yields four 32-bit words.
//
// Counter layout used throughout the library: (site, site >> 32, sweep,
// domain), except that the BOND domain counts pairs of rows (see below);
// key = (seed low word, seed high word).
#pragma once
#include <cstdint>

namespace xyk {

enum : uint32_t {
  kDomBond = 0,   // one draw per vertical pair of sites (counter m L + x):
                  // rows 2m / 2m+1 take words 0,1 / 2,3 as right, down; the
                  // right-bond word's bit 0 is the site's cluster coin
  kDomAxis = 1,   // the random axis of a sweep
  kDomInit = 2,   // random initial angles (sweep word 0xffffffff)
};

struct Words4 {
  uint32_t w0, w1, w2, w3;
};

__host__ __device__ __forceinline__ Words4 philox4x32_10(uint32_t c0,
                                                         uint32_t c1,
                                                         uint32_t c2,
                                                         uint32_t c3,
                                                         uint32_t k0,
                                                         uint32_t k1) {
  constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = static_cast<uint64_t>(kMul0) * c0;
    const uint64_t p1 = static_cast<uint64_t>(kMul1) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
    c1 = static_cast<uint32_t>(p1);
    c3 = static_cast<uint32_t>(p0);
    c0 = n0;
    c2 = n2;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  return Words4{c0, c1, c2, c3};
}

}  // namespace xyk
