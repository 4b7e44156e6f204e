// fock_sparse_mixed.cu -- instantiations of the any-sparsity H C kernel
// (fock_apply_sparse.cuh) for PolMixedP.
#include "fock_apply_sparse.cuh"

int fock_launch_sparse_mixed(const SparseArgs &sa, bool block, bool maps, int dev, cudaStream_t s) {
  return fock_launch_sparse_policy<PolMixedP, 8>(sa, block, maps, dev, s);
}
