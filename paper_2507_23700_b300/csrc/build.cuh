// Construction of the linear BVH (see build.cu).
#pragma once

#include "common.cuh"

namespace arbx {

// Atomic exchange with acquire-release semantics at device scope (the Apetrei
// handoff of the single-tree and forest builds): the caller's earlier stores
// are visible to a thread that later exchanges the same word, and that
// thread's later loads see them.
__device__ __forceinline__ int32_t exch_acq_rel(int32_t* p, int32_t v) {
  int32_t old;
  asm volatile("atom.acq_rel.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Device arrays of a built tree (owned by the arbx_tree_t that holds them).
struct BuiltTree {
  int64_t n = 0;
  int64_t nnodes = 0;        // internal nodes (n-1, or 1 pseudo node for n == 1)
  int32_t node_stride = 0;   // bytes per float32 node
  bool quantized = false;    // 16-bit nodes (QNode, or PNode when prel)
  bool prel = false;         // parent-relative 32-byte nodes (ARBX_PARENT_RELATIVE)
  void* nodes = nullptr;     // Node<D>[nnodes]
  QNode* qnodes = nullptr;   // 16-bit copy (3D, ARBX_QUANTIZED_NODES)
  PNode* pnodes = nullptr;   // parent-relative 16-bit copy (3D, with ARBX_PARENT_RELATIVE)
  float rframe[4] = {0, 0, 0, 0};  // PNode trees: frame of the root's box (host copy of a float4)
  TriLeaf* leaves = nullptr; // triangles: sorted leaf records
  void* wide = nullptr;      // Wide<D>[nnodes] (point and box trees)
  int32_t* leaf_orig = nullptr;  // quantized triangle trees: input index of each sorted leaf
  void* top[2] = {nullptr, nullptr};  // BFS copies of the top 255 / 1023 nodes
  int32_t ntop[2] = {0, 0};
  int32_t root = 0;          // internal index of the root
  float* scene = nullptr;    // device lo[dim], hi[dim]
  float scene_host[12];
};

// Build over n >= 1 primitives of `kind` and `dim` (data: device, row-major).
arbx_status build_tree(int kind, int dim, const float* data, int64_t n, uint32_t flags, BuiltTree* out,
                       cudaStream_t s);

}  // namespace arbx
