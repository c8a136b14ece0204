// Prints the host 1D tables of the CUDA path (mf_tables.cpp: GLL nodes, Gauss rule, S, D, Dc,
// 1D mass and stiffness, and the fast diagonalisation W, lam of (K, M)) for degrees 1..8, one
// "name n values..." line per array, for tests/test_host_tables.py to check against numpy and
// scipy.  Compiled as a host program together with mf_tables.cpp.
#include <cstdio>

#include "mf_internal.h"

static void put(const char* name, int k, const double* v, int rows, int cols, int ld) {
  std::printf("%s %d", name, k);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) std::printf(" %.17g", v[r * ld + c]);
  std::printf("\n");
}

int main() {
  for (int k = 1; k <= 8; ++k) {
    mf::HostTables t;
    if (mf::make_host_tables(k, &t) != 0) return 1;
    const int n = k + 1, L = mf::MAXN;
    put("nodes", k, t.nodes, 1, n, n);
    put("qx", k, t.qx, 1, n, n);
    put("qw", k, t.qw, 1, n, n);
    put("S", k, t.S, n, n, L);
    put("D", k, t.D, n, n, L);
    put("Dc", k, t.Dc, n, n, L);
    put("M", k, t.M, n, n, L);
    put("K", k, t.K, n, n, L);
    put("W", k, t.Wfd, n, n, L);
    put("lam", k, t.lam, 1, n, n);
  }
  return 0;
}
