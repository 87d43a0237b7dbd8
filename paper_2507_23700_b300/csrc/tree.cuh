// The tree handle behind the opaque arbx_tree of the C ABI.
#pragma once

#include "build.cuh"

struct arbx_tree_t {
  int device = 0;
  int32_t kind = ARBX_POINT;
  int32_t dim = 3;
  int64_t n = 0;
  uint32_t flags = 0;
  arbx::BuiltTree bt;
};
