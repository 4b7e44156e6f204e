// fock_twophase.cu -- instantiations of the two-phase dense-coefficient apply
// (fock_apply_twophase.cuh) for M = 2..8 orbitals.
#include "fock_apply_twophase.cuh"

template <int M>
static int launch_df(const TwoPhaseArgs &t, int dev, cudaStream_t s) {
  const ApplyArgs<uint32_t> &a = t.a;
  const TwoPhaseSmem<M> L(a.xdim, a.nsq, 2 * sizeof(float4), sizeof(TwoPhaseSlot) * M, FOCK_APPLY_THREADS);
  if (t.phases & 1) {
    const int st = fock_launch_grid(fock_twophase_x_df<M>, t, t.c_end - t.c_begin, L.total, dev, s);
    if (st) return st;
    if (t.phase1_done) FOCK_CUDA_TRY(cudaEventRecord(t.phase1_done, s));
  }
  if (!(t.phases & 2)) return FOCK_OK;
  return fock_launch_grid(fock_twophase_sigma_df<M>, t, (uint64_t)(t.g_end - t.g_begin) * a.nrhs, twophase_sigma_smem(a.rows, a.xdim, a.nsq),
                          dev, s);
}

template <int M>
static int launch_mixed(const TwoPhaseArgs &t, int dev, cudaStream_t s) {
  const ApplyArgs<uint32_t> &a = t.a;
  const TwoPhaseSmem<M> L(a.xdim, a.nsq, sizeof(float2), sizeof(TwoPhaseSlot) * M, FOCK_APPLY_THREADS);
  if (t.phases & 1) {
    const int st = fock_launch_grid(fock_twophase_x_mixed<M>, t, t.c_end - t.c_begin, L.total, dev, s);
    if (st) return st;
    if (t.phase1_done) FOCK_CUDA_TRY(cudaEventRecord(t.phase1_done, s));
  }
  if (!(t.phases & 2)) return FOCK_OK;
  return fock_launch_grid(fock_twophase_sigma_mixed<M>, t, (uint64_t)(t.g_end - t.g_begin) * a.nrhs,
                          twophase_sigma_smem(a.rows, a.xdim, a.nsq), dev, s);
}

int fock_launch_twophase(const TwoPhaseArgs &t, bool mixed, int dev, cudaStream_t s) {
  switch (t.a.M) {
#define FOCK_TP_CASE(MM) \
    case MM: return mixed ? launch_mixed<MM>(t, dev, s) : launch_df<MM>(t, dev, s);
    FOCK_TP_CASE(2)
    FOCK_TP_CASE(3)
    FOCK_TP_CASE(4)
    FOCK_TP_CASE(5)
    FOCK_TP_CASE(6)
    FOCK_TP_CASE(7)
    FOCK_TP_CASE(8)
#undef FOCK_TP_CASE
  }
  return FOCK_ERR_UNSUPPORTED;
}
