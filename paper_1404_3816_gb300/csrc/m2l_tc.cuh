// Tensor-core M2L of the H^2 product (internal).
#pragma once

#include "hikf_internal.cuh"

namespace hikf {

struct M2lTcArgs {
  int lev = 2, dim = 2, q = 0, ld = 0, sms = 1;
  int64_t box0 = 0, nbox = 0;         // first box of the level, boxes at the level
  const float* W = nullptr;           // [box][q][ld] multipoles (all levels)
  float* L = nullptr;                 // [box][q][ld] locals (all levels); written for this level
  const float* kop_level = nullptr;   // [offset][q][q] operators of this level
  const int64_t* nsrc = nullptr;      // per box (all levels): sources below
  const int64_t* npts = nullptr;      // per box (all levels): points below
  int* err = nullptr;                 // device word, set when a bounded wait times out
};

bool m2l_tc_supported(int q, int ld);
Status m2l_tc_level(const M2lTcArgs& a, cudaStream_t s);

}  // namespace hikf
