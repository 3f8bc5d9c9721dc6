// Known-answer source for Philox4x32-10 that is independent of this project:
// ATen's host Philox engine (an open-source header shipped with PyTorch).
// Reads "seed traj m" triples from stdin and prints the four 32-bit words of
// counter block m of subsequence traj under key seed.
#include <ATen/core/PhiloxRNGEngine.h>

#include <cinttypes>
#include <cstdio>

int main() {
  unsigned long long seed, traj, m;
  while (std::scanf("%llu %llu %llu", &seed, &traj, &m) == 3) {
    at::philox_engine eng(seed, traj, m);
    uint32_t w[4];
    for (int i = 0; i < 4; ++i) w[i] = eng();
    std::printf("%u %u %u %u\n", w[0], w[1], w[2], w[3]);
  }
  return 0;
}
