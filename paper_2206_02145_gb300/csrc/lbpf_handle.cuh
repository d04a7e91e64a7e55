// The simulation handle behind lbpf_t, shared by the files that implement the
// C ABI (lbpf_api.cu: create / step / read-out; surrogate.cu: the learned
// block propagator, which reads and replaces the state in place).
#pragma once

#include "../../include/lbpf.h"
#include "lbpf_internal.cuh"

struct lbpf {
  lbpf_params p;
  lbk::Model m;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  void* pops[2] = {nullptr, nullptr};
  void* phi[2] = {nullptr, nullptr};  // phi[cur] holds phi(t-1)
  int cur = 0;
  long long step = 0;
  bool initialized = false;
  unsigned* d_err = nullptr;
  double* d_partials = nullptr;
  double* d_diag = nullptr;  // [0..10] diag outputs, [16] solute total at init
  void* d_fields = nullptr;
  size_t fields_cap = 0;
  unsigned long long* d_facets = nullptr;  // facet-support results (first use)
  unsigned long long* h_facets = nullptr;  // their pinned host copy
  int facet_k = 0;             // normals of the enqueued measurement (0: none pending)
  double facet_nx[LBPF_MAX_FACETS], facet_ny[LBPF_MAX_FACETS];
  unsigned char* d_solid = nullptr;  // solid mask, px x ny bytes (first lbpf_set_solid)
  unsigned char* d_solid_tiles = nullptr;  // its per-tile flags
  int icx = 0, icy = 0, icz = 0;
  size_t dev_bytes = 0;
  size_t es = 4;  // population element bytes
  size_t rs = 4;  // phi ring element bytes
  lbk::StepMaps maps;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // graphs of shorter step counts (the remainder of an lbpf_step call below
  // the main graph's length), keyed by count and starting buffer parity
  static constexpr int kTailGraphs = 4;
  cudaGraphExec_t tail_graph[kTailGraphs] = {nullptr, nullptr, nullptr, nullptr};
  int tail_n[kTailGraphs] = {0, 0, 0, 0};
  int tail_parity[kTailGraphs] = {0, 0, 0, 0};
  int tail_next = 0;
  int status = LBPF_OK;
  int gen = 0;  // bumped whenever the state or the model constants are replaced
  char msg[256] = {0};
};
