// fock_apply_mixed.cu -- instantiations of the H C kernel for PolMixed
// (one translation unit per arithmetic policy so the build compiles them in
// parallel).
#include "fock_apply_kernel.cuh"

namespace {
template <class Idx, bool MAPS>
int by_shape(const ApplyArgs<Idx> &a, int maxm, bool nrhs16, int dev, cudaStream_t s) {
  switch (maxm) {
    case 4:
      return nrhs16 ? fock_launch_list<Idx, 4, PolMixed, 16, MAPS>(a, dev, s)
                    : fock_launch_list<Idx, 4, PolMixed, 1, MAPS>(a, dev, s);
    case 8:
      return nrhs16 ? fock_launch_list<Idx, 8, PolMixed, 16, MAPS>(a, dev, s)
                    : fock_launch_list<Idx, 8, PolMixed, 1, MAPS>(a, dev, s);
    case 12:
      return nrhs16 ? fock_launch_list<Idx, 12, PolMixed, 16, MAPS>(a, dev, s)
                    : fock_launch_list<Idx, 12, PolMixed, 1, MAPS>(a, dev, s);
  }
  return FOCK_ERR_UNSUPPORTED;
}

template <bool MAPS>
int by_shape64(const ApplyArgs<uint64_t> &a, int maxm, int dev, cudaStream_t s) {
  switch (maxm) {
    case 4: return fock_launch_list<uint64_t, 4, PolMixed, 1, MAPS>(a, dev, s);
    case 8: return fock_launch_list<uint64_t, 8, PolMixed, 1, MAPS>(a, dev, s);
    case 12: return fock_launch_list<uint64_t, 12, PolMixed, 1, MAPS>(a, dev, s);
  }
  return FOCK_ERR_UNSUPPORTED;
}
}  // namespace

int fock_launch_apply_mixed(const void *args, bool idx32, int maxm, bool nrhs16, bool maps,
                        int dev, cudaStream_t s) {
  if (idx32) {
    const auto &a = *(const ApplyArgs<uint32_t> *)args;
    return maps ? by_shape<uint32_t, true>(a, maxm, nrhs16, dev, s)
                : by_shape<uint32_t, false>(a, maxm, nrhs16, dev, s);
  }
  if (maps || nrhs16) return FOCK_ERR_UNSUPPORTED;
  return by_shape64<false>(*(const ApplyArgs<uint64_t> *)args, maxm, dev, s);
}
