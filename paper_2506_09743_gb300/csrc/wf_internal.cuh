// Host-side definition of the opaque qmc_wf handle, shared by the C ABI
// translation units (capi.cu, server.cu).
#pragma once

#include <mutex>
#include <string>
#include <vector>

#include "qmc_internal.cuh"

namespace qmc {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace qmc

// Records msg as the calling thread's qmc_last_error() text and returns s.
qmc_status set_error(qmc_status s, const std::string& msg);

// Host copy of the inputs of qmc_create_wf (parameters are updated in place by
// qmc_set_params, geometry by qmc_set_geometry; the device tables are rebuilt
// from it).
struct HostSpec {
  int na = 0, nup = 0, ndn = 0, nao = 0, nmo = 0, ndet = 0;
  std::vector<double> xyz, z;
  std::vector<int> ao_atom, ao_kind, ao_pow, prim_start;
  std::vector<double> prim_exp, prim_coef, mo, det_w;
  std::vector<int> det_exc;
  double w0p = 0.25, w0a = 0.5, b = 1.0, w = 0.0;
  std::vector<double> jen;   // [3] or empty: electron-nucleus Jastrow kernel
  std::vector<double> jeen;  // [n][7]: electron-electron-nucleus terms
};

struct qmc_wf {
  int device = 0;
  int precision = QMC_FP64;
  HostSpec spec;
  qmc::WfDev dev{};
  // energy-gradient scratch (library-owned)
  void* gws = nullptr;
  size_t gws_bytes = 0;
  // device allocations
  void* blob = nullptr;
  // library-owned workspace and host-call staging buffers
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* stage = nullptr;
  size_t stage_bytes = 0;
  // optional per-stage timing events
  bool timing = false;
  bool timed_once = false;
  cudaEvent_t tev[6] = {};  // Jastrow, AO+MO, det (start, end)
  int det_method = QMC_DET_TABLE;
  cudaStream_t cap_stream = nullptr;  // capture stream of the Metropolis step graph
  // bounded device waits: budget in SM cycles (about 1 s at 2 GHz), the
  // sticky status word their kernels set when one gives up (qmc_check_status)
  // and a page-locked host word the status is read into
  long long wait_cycles = 1ll << 31;
  int* err_wf = nullptr;
  int* status_host = nullptr;
  std::mutex mu;
};

// qmc_sample / qmc_local_energy with the choice of clearing the workspace's
// status word first (reset = true, the public calls) or keeping it (the
// server clears it once per request and reads it when the request retires)
qmc_status sample_call(qmc_wf* wf, double* walkers, int64_t n_walkers, int64_t ldw, int32_t n_steps, double step,
                       uint64_t seed, uint64_t first_walker, uint64_t step_offset, double* log_psi, int64_t* n_accept,
                       void* workspace, size_t workspace_bytes, void* stream, bool reset);
qmc_status local_energy_call(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* e_loc,
                             double* log_psi, void* workspace, size_t workspace_bytes, void* stream, bool reset);
// the status word inside a workspace of qmc_workspace_size(wf, n_walkers) bytes
int* workspace_status(const qmc_wf* wf, void* workspace, int64_t n_walkers);
