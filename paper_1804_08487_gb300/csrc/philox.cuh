// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
// Random Numbers: As Easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64
// multiplications with Weyl-sequence key updates.  Key words are the low and
// high halves of the 64-bit seed.
#pragma once
#include <cstdint>

namespace cb {

struct Philox4 {
  uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint64_t seed) {
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c0;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
    c1 = static_cast<uint32_t>(p1);
    c3 = static_cast<uint32_t>(p0);
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return {c0, c1, c2, c3};
}

// The key words of the ten rounds for one seed: ks[2r], ks[2r + 1] = the
// key after r Weyl increments.
__host__ __device__ inline void philox_round_keys(uint64_t seed, uint32_t* ks) {
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    ks[2 * r] = k0;
    ks[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// philox4x32_10 with the round keys given (philox_round_keys of the seed).
// A kernel that draws under one seed takes them as a kernel parameter: each
// round's key words are then constant-bank operands, not two additions.
__device__ __forceinline__ Philox4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                    const uint32_t* ks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c0;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ ks[2 * r];
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ ks[2 * r + 1];
    c1 = static_cast<uint32_t>(p1);
    c3 = static_cast<uint32_t>(p0);
    c0 = n0;
    c2 = n2;
  }
  return {c0, c1, c2, c3};
}

// Permutation key of node x in super step g: counter (x, 0, g, 0), words 0-1.
__device__ __forceinline__ uint64_t node_key(uint64_t seed, uint32_t x, uint32_t g) {
  const Philox4 r = philox4x32_10(x, 0u, g, 0u, seed);
  return (static_cast<uint64_t>(r.w0) << 32) | r.w1;
}

// Shuffle key of the edge identified by step-start positions lo < hi, for the
// trade that owns position lo (words 0-1) or position hi (words 2-3).
__device__ __forceinline__ uint64_t edge_key(uint64_t seed, uint32_t lo, uint32_t hi, uint32_t g,
                                             bool lo_side) {
  const Philox4 r = philox4x32_10(lo, hi, g, 1u, seed);
  return lo_side ? ((static_cast<uint64_t>(r.w0) << 32) | r.w1)
                 : ((static_cast<uint64_t>(r.w2) << 32) | r.w3);
}

}  // namespace cb
