// fock_sparse_f64.cu -- instantiations of the any-sparsity H C kernel
// (fock_apply_sparse.cuh) for PolF64.
#include "fock_apply_sparse.cuh"

int fock_launch_sparse_f64(const SparseArgs &sa, bool block, bool maps, int dev, cudaStream_t s) {
  return fock_launch_sparse_policy<PolF64, 4>(sa, block, maps, dev, s);
}
