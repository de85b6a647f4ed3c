// stm_probe.cu -- test infrastructure: prints, on the host, the structural
// sparsity mask of the interval STM that the compiled model declares
// (model_stm_row_mask), the visiting order the PIPG steps derive from it and
// the offsets of the compact block storage (make_stm_order), for
// tests/test_stm_mask.py to check against the oracle.
#include <cstdio>

#include "pdg_device.cuh"

using namespace pdg;

int main() {
  constexpr StmOrder S = make_stm_order();
  std::printf("NX %d\n", NX);
  for (int i = 0; i < NX; ++i) std::printf("mask %d %u\n", i, model_stm_row_mask(i));
  for (int a = 0; a < NX; ++a)
    std::printf("order %d %d %d %d %d %llu %llu\n", a, S.row_order[a], S.col_order[a], S.row_nnz[a], S.col_nnz[a],
                S.row_list[a], S.col_list[a]);
  std::printf("compact %d %d\n", S.nnz, STM_SAS);
  for (int a = 0; a < NX; ++a)
    std::printf("offsets %d %d %llu %llu %llu %llu\n", a, S.row_start[a], S.row_off[a][0], S.row_off[a][1],
                S.col_off[a][0], S.col_off[a][1]);
  return 0;
}
