// fock_sparse_df.cu -- instantiations of the any-sparsity H C kernel
// (fock_apply_sparse.cuh) for PolDFP.
#include "fock_apply_sparse.cuh"

int fock_launch_sparse_df(const SparseArgs &sa, bool block, bool maps, int dev, cudaStream_t s) {
  return fock_launch_sparse_policy<PolDFP, 4>(sa, block, maps, dev, s);
}
