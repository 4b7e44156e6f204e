// fock_dense_mixed.cu -- instantiations of the dense-coefficient H C kernel
// (fock_apply_dense.cuh) for M = 1..10 orbitals.
#include "fock_apply_dense.cuh"

template <int M>
static int launch_m(const ApplyArgs<uint32_t> &a, bool block, bool maps, int dev, cudaStream_t s) {
  const DenseSmem<M> L(a.xdim, a.nsq, sizeof(float2));
  if (maps) return fock_launch_dense(fock_apply_dense_mixed<M, 1, true>, a, L.total, dev, s);
  if (block) return fock_launch_dense(fock_apply_dense_mixed<M, 8, false>, a, L.total, dev, s);
  return fock_launch_dense(fock_apply_dense_mixed<M, 1, false>, a, L.total, dev, s);
}

int fock_launch_dense_mixed(const ApplyArgs<uint32_t> &a, bool block, bool maps, int dev, cudaStream_t s) {
  if (maps && block) return FOCK_ERR_UNSUPPORTED;
  switch (a.M) {
    case 1: return launch_m<1>(a, block, maps, dev, s);
    case 2: return launch_m<2>(a, block, maps, dev, s);
    case 3: return launch_m<3>(a, block, maps, dev, s);
    case 4: return launch_m<4>(a, block, maps, dev, s);
    case 5: return launch_m<5>(a, block, maps, dev, s);
    case 6: return launch_m<6>(a, block, maps, dev, s);
    case 7: return launch_m<7>(a, block, maps, dev, s);
    case 8: return launch_m<8>(a, block, maps, dev, s);
    case 9: return launch_m<9>(a, block, maps, dev, s);
    case 10: return launch_m<10>(a, block, maps, dev, s);
  }
  return FOCK_ERR_UNSUPPORTED;
}
