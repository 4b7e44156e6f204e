// fock_noalloc.cu -- sigma = H C without any device allocation.
//
// The FP64-class apply (FOCK_PREC_F64) needs device scratch: a header of
// status words and a hi/lo split copy of C.  fock_apply_H takes that scratch
// from the caller or allocates it on first use.  Some callers can do neither:
// a caller whose device memory belongs to another allocator (a caching
// allocator or a fixed pool it must not bypass), or one running in a loop where
// a cudaMalloc/cudaFree would synchronise the device and stall its other
// streams.  fock_apply_H_noalloc serves them from a fixed array in the
// library's own device image instead.
//
// The array is a file-scope __device__ object of FOCK_NOALLOC_SCRATCH_BYTES.
// Host code cannot use the array's name as a device address, so the address
// is looked up with cudaGetSymbolAddress once per device (with that device
// current) and cached.  With CUDA's lazy module loading the look-up is what
// loads this module on a device, which creates the array there (a device
// allocation by the driver, and possibly a synchronisation).  fock_space_create
// therefore performs the look-up for its device, so that the no-alloc calls
// on a space never trigger it.
#include <mutex>

#include "fock_common.cuh"

static __device__ __align__(256) unsigned char fock_noalloc_scratch_array[FOCK_NOALLOC_SCRATCH_BYTES];

namespace {
const int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];
}  // namespace

int fock_noalloc_scratch(int dev, void **addr) {
  if (dev < 0 || dev >= kMaxDevices) return FOCK_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, fock_noalloc_scratch_array);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return FOCK_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *addr = g_addr[dev];
  return FOCK_OK;
}

extern "C" int fock_apply_H_noalloc(const fock_space *sp, const fock_ham *ham, const void *C_dev,
                                    void *sigma_dev, int32_t nrhs, int arm, void *stream) {
  if (!sp || !ham || ham->sp != sp || !C_dev || !sigma_dev) return FOCK_ERR_ARG;
  if (nrhs < 1 || nrhs > FOCK_MAX_NRHS) return FOCK_ERR_ARG;
  if (arm < FOCK_ARM_AUTO || arm > FOCK_ARM_MAPS) return FOCK_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FOCK_ERR_CUDA;
  if (dev != sp->device) return FOCK_ERR_DEVICE;
  const size_t need = fock_apply_ws_bytes(sp, ham, nrhs, FOCK_PREC_F64);
  if (need > (size_t)FOCK_NOALLOC_SCRATCH_BYTES) return FOCK_ERR_SCRATCH_LIMIT;
  void *scratch = nullptr;
  const int st = fock_noalloc_scratch(dev, &scratch);
  if (st) return st;
  // The apply clears the status words it needs at the start of every call and
  // overwrites the whole split copy, so nothing left by an earlier call is read.
  return fock_apply_internal(sp, ham, C_dev, sigma_dev, nrhs, FOCK_PREC_F64, arm, scratch,
                             (size_t)FOCK_NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream);
}
