// Prints the host-built sweep tables of one sector as plain text, for the
// CPU test tests/test_host_tables.py (which checks them against the string
// enumeration of the oracle).  Usage: host_tables_driver N n W
//
// Output:
//   W <W> npos <npos>
//   orbit <a> <m> <clo> <RO> <addr_0> ... <addr_{C(W,m)-1}>   (one line per item,
//   pad <a>                                                   in list order)
//   pass <q0> <q1> <q2> <q3> <keep>
//   rec <m> <gbits> <flips> <addr_0> ... <addr_{C(4,m)-1}>    (in list order)
//   rpad
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "fs_internal.h"

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const int N = atoi(argv[1]), n = atoi(argv[2]), W = atoi(argv[3]);
  std::vector<uint32_t> orbits;
  std::vector<int> off;
  std::vector<uint16_t> offs;
  std::vector<uint8_t> okey;
  fs::window_tables_host(N, n, W, orbits, off, offs, okey);
  const int npos = N - W + 1;
  printf("W %d npos %d\n", W, npos);
  for (int a = 0; a < npos; ++a)
    for (int i = off[a]; i < off[a + 1]; ++i) {
      const uint32_t d = orbits[i];
      const int m = (int)(d >> 24);
      if (m == 0) {
        printf("pad %d\n", a);
        continue;
      }
      const int RO = d & 0xFFFF, clo = (d >> 16) & 0xFF;
      printf("orbit %d %d %d %d", a, m, clo, RO);
      for (int S = 0; S < (1 << W); ++S)
        if (__builtin_popcount(S) == m)
          printf(" %d", RO + offs[(((size_t)a * (n + 1) + clo) << W) + S]);
      printf("\n");
    }
  std::vector<fs::TPass> passes;
  std::vector<fs::TRecord> recs;
  std::vector<uint8_t> rkey;
  fs::tpass_tables_host(N, n, passes, recs, rkey);
  for (const auto& p : passes) {
    printf("pass %d %d %d %d %u\n", p.q[0], p.q[1], p.q[2], p.q[3], p.keep);
    for (int i = p.rec0; i < p.rec1; ++i) {
      const fs::TRecord& r = recs[i];
      if (r.m == 0) {
        printf("rpad\n");
        continue;
      }
      int ns = 0;
      for (int s = 0; s < 16; ++s) ns += __builtin_popcount(s) == r.m;
      printf("rec %d %d %d", r.m, r.gbits, r.flips);
      for (int k = 0; k < ns; ++k) printf(" %d", r.addr[k]);
      printf("\n");
    }
  }
  return 0;
}
