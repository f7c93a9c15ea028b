// Launch geometry of the fast-diagonalization passes (shared by the kernel
// and the host code that sets it up).
#pragma once

namespace rk {

struct FdmGeo {
  int n;        // nodes per direction
  int rows;     // n*n
  int nt;       // N columns, a multiple of 16: all of Q (n <= 128), or both CTAs' halves together (pair, <= 256)
  int kblocks;  // 128-byte K blocks: ceil(n * sizeof(S) / 128)
  int mtiles;   // ceil(rows / 128) (pair: ceil(rows / 256))
  int pair;     // 1: fdm_pass_pair on CTA pairs (n > 128)
  int stages;   // X stages in the TMA ring (as many as shared memory holds, <= 6)
};

}  // namespace rk
