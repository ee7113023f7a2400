// Batched translation of several independent plans (uneven grids, ranks and
// RHS counts).  The instances that the batch mode of the kernels covers
// (batch_persistent_ok) run together, one launch per phase and shape class
// (batch_launch.cu); any other instance runs its own launch sequence on one
// of a few side streams.  Repeated calls with the same buffers replay one
// captured CUDA graph.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fmmfft.h"
#include "plan_internal.h"

struct fmmfft_batch_s {
  std::vector<fmmfft_plan> plans;
  std::vector<cudaStream_t> side;       // fork streams
  std::vector<cudaEvent_t> joined;      // one per side stream
  cudaEvent_t forked = nullptr;
  // the last call's arguments and, once they repeat, its captured graph
  std::vector<const void*> key_in;
  std::vector<void*> key_out;
  std::vector<int> key_nrhs;
  int key_seen = 0;                     // consecutive calls with this key
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  fmm::BatchDev dev;                    // descriptors of the persistent launches
  int persistent = 1;                   // 0: every instance on its own launches
  int shared_last = 0;                  // instances in the shared launches of the last call
};

namespace {

constexpr int kSideStreams = 4;

void drop_graph(fmmfft_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Fork from `stream`: the shared launches of the instances they cover on
// `stream`, every other instance on a side stream; join back.
int launch_all(fmmfft_batch_s* b, const void* const* in, void* const* out, const int* nrhs,
               const std::vector<void*>& inter, const std::vector<size_t>& cap, cudaStream_t stream) {
  if (cudaEventRecord(b->forked, stream) != cudaSuccess) return FMMFFT_ERR_CUDA;
  for (auto s : b->side)
    if (cudaStreamWaitEvent(s, b->forked, 0) != cudaSuccess) return FMMFFT_ERR_CUDA;
  std::vector<fmm::TranslateArgs> together;
  std::vector<size_t> alone;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    fmm::TranslateArgs a;
    const int st = fmm::translate_args_for(b->plans[i], in[i], out[i], nrhs[i], inter[i], cap[i], &a);
    if (st != FMMFFT_OK) return st;
    if (b->persistent && fmm::batch_persistent_ok(a)) {
      a.stream = stream;
      together.push_back(a);
    } else {
      alone.push_back(i);
    }
  }
  b->shared_last = (int)together.size();
  if (!together.empty() && fmm::launch_translate_batch(together, b->dev, stream, b->side) != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  for (size_t k = 0; k < alone.size(); ++k) {
    const size_t i = alone[k];
    const int st = fmm::translate_into(b->plans[i], in[i], out[i], nrhs[i], b->side[k % b->side.size()],
                                       inter[i], cap[i]);
    if (st != FMMFFT_OK) return st;
  }
  for (size_t k = 0; k < b->side.size(); ++k) {
    if (cudaEventRecord(b->joined[k], b->side[k]) != cudaSuccess) return FMMFFT_ERR_CUDA;
    if (cudaStreamWaitEvent(stream, b->joined[k], 0) != cudaSuccess) return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

}  // namespace

extern "C" {

int fmmfft_batch_create(fmmfft_batch* out, const fmmfft_plan* plans, int nplans) {
  if (!out || !plans || nplans < 1) return FMMFFT_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < nplans; ++i)
    if (!plans[i]) return FMMFFT_ERR_INVALID_ARG;
  fmmfft_batch_s* b = new (std::nothrow) fmmfft_batch_s();
  if (!b) return FMMFFT_ERR_OOM;
  b->plans.assign(plans, plans + nplans);
  const char* sep = std::getenv("FMMFFT_BATCH_SEPARATE");
  b->persistent = (sep && *sep && std::strcmp(sep, "0") != 0) ? 0 : 1;
  const int ns = nplans < kSideStreams ? nplans : kSideStreams;
  b->side.assign(ns, nullptr);
  b->joined.assign(ns, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < ns; ++k)
    ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->joined[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    fmmfft_batch_destroy(b);
    return FMMFFT_ERR_CUDA;
  }
  *out = b;
  return FMMFFT_OK;
}

int fmmfft_batch_translate(fmmfft_batch b, const void* const* S_in, void* const* S_out, const int* nrhs,
                           void* stream) {
  if (!b || !S_in || !S_out || !nrhs) return FMMFFT_ERR_INVALID_ARG;
  const size_t n = b->plans.size();
  cudaStream_t s = (cudaStream_t)stream;
  // every instance's intermediate exists before anything is launched or
  // captured (an allocation would synchronise)
  std::vector<void*> inter(n);
  std::vector<size_t> cap(n);
  for (size_t i = 0; i < n; ++i) {
    if (!S_in[i] || !S_out[i]) return FMMFFT_ERR_INVALID_ARG;
    const int st = fmm::plan_intermediate(b->plans[i], nrhs[i], stream, &inter[i], &cap[i]);
    if (st != FMMFFT_OK) return st;
  }
  const bool same = b->key_in.size() == n &&
                    std::equal(b->key_in.begin(), b->key_in.end(), S_in) &&
                    std::equal(b->key_out.begin(), b->key_out.end(), S_out) &&
                    std::equal(b->key_nrhs.begin(), b->key_nrhs.end(), nrhs);
  int st = FMMFFT_OK;
  if (same && b->exec) {
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) st = FMMFFT_ERR_CUDA;
  } else if (same && b->key_seen >= 1 && s != nullptr) {
    // second call with the same arguments: capture once, replay from now on
    drop_graph(b);
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return FMMFFT_ERR_CUDA;
    }
    st = launch_all(b, S_in, S_out, nrhs, inter, cap, s);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st == FMMFFT_OK && (e != cudaSuccess || !g)) st = FMMFFT_ERR_CUDA;
    if (st == FMMFFT_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = FMMFFT_ERR_CUDA;
    b->graph = g;
    if (st == FMMFFT_OK && cudaGraphLaunch(b->exec, s) != cudaSuccess) st = FMMFFT_ERR_CUDA;
    if (st != FMMFFT_OK) {
      cudaGetLastError();
      drop_graph(b);
    }
  } else {
    st = launch_all(b, S_in, S_out, nrhs, inter, cap, s);
  }
  if (!same) {
    drop_graph(b);
    b->key_in.assign(S_in, S_in + n);
    b->key_out.assign(S_out, S_out + n);
    b->key_nrhs.assign(nrhs, nrhs + n);
    b->key_seen = 0;
  }
  b->key_seen += 1;
  for (auto p : b->plans) fmm::plan_set_last_stream(p, stream);
  return st;
}

int fmmfft_batch_autotune(fmmfft_batch b, const int* nrhs, double budget_ms) {
  if (!b || !nrhs || !(budget_ms > 0)) return FMMFFT_ERR_INVALID_ARG;
  const double each = budget_ms / (double)b->plans.size();
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const int st = fmmfft_autotune(b->plans[i], nrhs[i], each);
    if (st != FMMFFT_OK) return st;
  }
  // schedules changed: the captured graph no longer matches
  drop_graph(b);
  b->key_in.clear();
  b->key_out.clear();
  b->key_nrhs.clear();
  b->key_seen = 0;
  return FMMFFT_OK;
}

int fmmfft_batch_shared_count(fmmfft_batch b, int* count) {
  if (!b || !count) return FMMFFT_ERR_INVALID_ARG;
  *count = b->shared_last;
  return FMMFFT_OK;
}

int fmmfft_batch_destroy(fmmfft_batch b) {
  if (!b) return FMMFFT_ERR_INVALID_ARG;
  for (auto s : b->side)
    if (s) cudaStreamSynchronize(s);
  drop_graph(b);
  for (auto s : b->side)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->joined)
    if (e) cudaEventDestroy(e);
  if (b->forked) cudaEventDestroy(b->forked);
  fmm::batch_dev_release(b->dev);
  delete b;
  return FMMFFT_OK;
}

}  // extern "C"
