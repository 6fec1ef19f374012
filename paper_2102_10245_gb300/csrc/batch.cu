// Batched MTTKRP: many (tensor, mode) MTTKRPs of uneven order and size in
// one CUDA graph.  Items are grouped by kernel shape (order, key words, rank,
// accumulation variant); every group runs as one persistent launch over a
// device work list of its items' thread-block units, so small tensors share
// the GPU instead of each occupying a launch.  Items whose shape has no
// specialised kernel run on their own inside the same graph.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "mttkrp_kernels.cuh"

struct alto_batch_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> bufs;  // device buffers the plan owns (cudaMalloc)
  int items = 0;
  int groups = 0;
  int single = 0;
  int kernels = 0;  // kernel nodes in the graph
};

namespace alto {

alto_status check_mttkrp_args(const alto_tensor_s* t, int mode, const void* const* factors, int R,
                              alto_dtype fdtype, const void* out, int variant);
int resolve_variant(const alto_tensor_s* t, int mode, int R, size_t osz, int variant);
void fill_launch(const alto_tensor_s* t, int mode, const void* const* factors, int R, void* out,
                 MttkrpLaunch* l);
int64_t mttkrp_parts(const alto_tensor_s* t, int mode, int variant);
size_t smem_temp_bytes(const alto_tensor_s* t, int mode, int R, size_t osz, int* rows_out);
cudaError_t mttkrp_launch(alto_tensor_s* t, int mode, const void* const* factors, int R,
                          alto_dtype fdtype, void* out, int variant, size_t osz, cudaStream_t s);

namespace {

// the input factors of a mode-`mode` MTTKRP in kernel slot order
std::vector<const void*> factors_in_slot_order(const alto_tensor_s* t, int mode, const void* const* f) {
  std::vector<const void*> r;
  for (int m = 0; m < t->lay.N; ++m)
    if (m != mode) r.push_back(f[m]);
  return r;
}

constexpr int kBatchHotReplicas = 8;
constexpr int kBatchHotCap = 256;
constexpr size_t kBatchBranches = 16;  // parallel branches of the graph

void free_plan(alto_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void* p : b->bufs) cudaFree(p);
  b->bufs.clear();
  b->exec = nullptr;
  b->graph = nullptr;
}

template <typename T>
T* upload(alto_batch_s* b, const std::vector<T>& v, cudaError_t* err) {
  void* p = nullptr;
  *err = cudaMalloc(&p, sizeof(T) * (v.empty() ? 1 : v.size()));
  if (*err != cudaSuccess) return nullptr;
  b->bufs.push_back(p);
  if (!v.empty()) *err = cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return static_cast<T*>(p);
}

}  // namespace

}  // namespace alto

using namespace alto;

extern "C" {

alto_status alto_batch_create(alto_batch_t* out, int count, const alto_t* tensors, const int* modes,
                              const void* const* const* factors, const int* ranks, alto_dtype fdtype,
                              void* const* outs, const int* variants, void* stream) {
  if (out == nullptr) return fail(ALTO_EINVAL, "null output");
  *out = nullptr;
  if (count < 0 || (count > 0 && (tensors == nullptr || modes == nullptr || factors == nullptr ||
                                  ranks == nullptr || outs == nullptr)))
    return fail(ALTO_EINVAL, "bad batch arguments");
  const size_t osz = fdtype == ALTO_F64 ? 8 : 4;
  const size_t fsz = fdtype == ALTO_F64 ? 8 : (fdtype == ALTO_F32 ? 4 : 2);
  for (int i = 0; i < count; ++i) {
    if (tensors[i] == nullptr) return fail(ALTO_EINVAL, "item %d: null tensor", i);
    const int v = variants ? variants[i] : ALTO_VAR_AUTO;
    const alto_status st = check_mttkrp_args(tensors[i], modes[i], factors[i], ranks[i], fdtype, outs[i], v);
    if (st != ALTO_OK) return st;
  }
  alto_batch_s* b = new alto_batch_s();
  b->items = count;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;

  // item descriptions, grouped by kernel shape
  using Key = std::tuple<int, int, int, int, int>;  // N, stored key words, R, variant, fused body
  struct Zero {
    void* p;
    size_t bytes;
  };
  struct HostGroup {
    std::vector<MttkrpArgs> items;
    std::vector<Zero> zeros;  // outputs and hot-row replicas of the items
    size_t smem = 0;
    double cost = 0;          // estimated work: streamed and gathered bytes
  };
  std::map<Key, HostGroup> groups;
  std::vector<int> single;    // items run on their own
  std::vector<Zero> empty_zeros;
  std::vector<HotItem> hot_items;
  std::vector<int64_t> hot_prefix(1, 0);
  for (int i = 0; i < count; ++i) {
    alto_tensor_s* t = tensors[i];
    const int mode = modes[i], R = ranks[i];
    const Zero z{outs[i], static_cast<size_t>(t->lay.dims[mode]) * R * osz};
    if (t->M == 0) {
      empty_zeros.push_back(z);
      continue;
    }
    int v = resolve_variant(t, mode, R, osz, variants ? variants[i] : ALTO_VAR_AUTO);
    if (v == ALTO_VAR_TEMP) v = ALTO_VAR_WARPAGG;  // the per-unit device Temp is not batched
    if (!mttkrp_specialised(t->lay.N, R) || v == ALTO_VAR_GENERIC) {
      single.push_back(i);
      continue;
    }
    const int fused = (v == ALTO_VAR_ATOMIC || v == ALTO_VAR_WARPAGG) &&
                      fused_ok(t->lay.N, R, fsz, factors_in_slot_order(t, mode, factors[i]).data(), outs[i], osz,
                               t->lay.dims[mode]);
    const Key key{t->lay.N, t->lay.CW, R, v, fused};
    HostGroup& hg = groups[key];
    hg.zeros.push_back(z);
    hg.cost += static_cast<double>(t->M) * (4.0 * t->lay.CW + 4.0 + (t->lay.N - 1) * R * fsz) +
               static_cast<double>(z.bytes);
    MttkrpLaunch l{};
    fill_launch(t, mode, factors[i], R, outs[i], &l);
    l.args.L = mttkrp_parts(t, mode, v);
    size_t smem = 0;
    if (v == ALTO_VAR_SMEM) {
      int rows = 0;
      smem = smem_temp_bytes(t, mode, R, osz, &rows);
      l.args.smem_rows = rows;
    }
    if (v == ALTO_VAR_WARPAGG && t->lay.dims[mode] <= (1ull << 31) && t->hot_n[mode] > 0) {
      const int H = t->hot_n[mode] < kBatchHotCap ? t->hot_n[mode] : kBatchHotCap;
      int bits = 1;
      while ((1 << bits) < 2 * H) ++bits;
      void* rep = nullptr;
      const size_t bytes = static_cast<size_t>(kBatchHotReplicas) * H * R * osz;
      e = cudaMalloc(&rep, bytes);
      if (e != cudaSuccess) break;
      b->bufs.push_back(rep);
      hg.zeros.push_back({rep, bytes});
      l.args.hot = t->hot[mode];
      l.args.hot_n = H;
      l.args.hot_bits = bits;
      l.args.hot_key_bit = t->lay.hot_bit[mode];
      l.args.hot_rep = rep;
      smem = static_cast<size_t>(2) * (1u << bits) * sizeof(uint32_t);
      hot_items.push_back({rep, t->hot[mode], outs[i], H, R, kBatchHotReplicas, 0});
      hot_prefix.push_back(hot_prefix.back() + static_cast<int64_t>(H) * R);
    }
    hg.items.push_back(l.args);
    hg.smem = std::max(hg.smem, smem);
  }

  // device work lists, largest group first
  struct Group {
    Key key;
    const HostGroup* host;
    MttkrpArgs* items;
    int64_t* prefix;
    int64_t units;
  };
  std::vector<Group> dev_groups;
  if (e == cudaSuccess) {
    for (auto& kv : groups) {
      std::vector<int64_t> prefix(1, 0);
      for (const MttkrpArgs& a : kv.second.items) prefix.push_back(prefix.back() + (a.L + kUnitSegs - 1) / kUnitSegs);
      Group g{kv.first, &kv.second, nullptr, nullptr, prefix.back()};
      g.items = upload(b, kv.second.items, &e);
      if (e != cudaSuccess) break;
      g.prefix = upload(b, prefix, &e);
      if (e != cudaSuccess) break;
      dev_groups.push_back(g);
    }
    std::sort(dev_groups.begin(), dev_groups.end(),
              [](const Group& x, const Group& y) { return x.host->cost > y.host->cost; });
  }
  HotItem* d_hot = nullptr;
  int64_t* d_hot_prefix = nullptr;
  if (e == cudaSuccess && !hot_items.empty()) {
    d_hot = upload(b, hot_items, &e);
    if (e == cudaSuccess) d_hot_prefix = upload(b, hot_prefix, &e);
  }
  if (e != cudaSuccess) {
    free_plan(b);
    delete b;
    return fail(ALTO_ECUDA, "batch plan: %s", cudaGetErrorString(e));
  }

  // Capture: the groups (their zeroing, then their persistent launch, the
  // costliest first) and the stand-alone items run on parallel branches of
  // the graph; the hot-row reduction follows once every branch is done.
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int branches = static_cast<int>(std::min<size_t>(kBatchBranches, dev_groups.size() + single.size()));
  std::vector<cudaStream_t> fs(branches, nullptr);
  std::vector<cudaEvent_t> join(branches, nullptr);
  cudaEvent_t fork = nullptr;
  cudaStream_t own = nullptr;  // the legacy default stream cannot be captured
  if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) {
    e = cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking);
    s = own;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int k = 0; e == cudaSuccess && k < branches; ++k) {
    e = cudaStreamCreateWithFlags(&fs[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
  }
  const uint64_t launches0 = launch_total();
  bool capturing = false;
  if (e == cudaSuccess) {
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    capturing = e == cudaSuccess;
  }
  for (size_t z = 0; e == cudaSuccess && z < empty_zeros.size(); ++z)
    e = cudaMemsetAsync(empty_zeros[z].p, 0, empty_zeros[z].bytes, s);
  if (e == cudaSuccess && branches > 0) e = cudaEventRecord(fork, s);
  for (int k = 0; e == cudaSuccess && k < branches; ++k) e = cudaStreamWaitEvent(fs[k], fork, 0);
  for (size_t gi = 0; e == cudaSuccess && gi < dev_groups.size(); ++gi) {
    const Group& g = dev_groups[gi];
    cudaStream_t bs = fs[gi % branches];
    for (size_t z = 0; e == cudaSuccess && z < g.host->zeros.size(); ++z)
      e = cudaMemsetAsync(g.host->zeros[z].p, 0, g.host->zeros[z].bytes, bs);
    if (e != cudaSuccess) break;
    BatchLaunch bl{};
    bl.args.items = g.items;
    bl.args.unit_prefix = g.prefix;
    bl.args.nitems = static_cast<int>(g.host->items.size());
    bl.args.hot_replicas = kBatchHotReplicas;
    bl.N = std::get<0>(g.key);
    bl.W32 = std::get<1>(g.key);
    bl.R = std::get<2>(g.key);
    bl.variant = std::get<3>(g.key);
    bl.sms = sms;
    bl.smem_dyn = g.host->smem;
    bl.units = g.units;
    bl.fused = std::get<4>(g.key) != 0;
    e = mttkrp_batch_dispatch(bl, fdtype, bs);
  }
  for (size_t k = 0; e == cudaSuccess && k < single.size(); ++k) {
    const int i = single[k];
    // no specialised kernel (or the generic one requested): the generic kernel
    e = mttkrp_launch(tensors[i], modes[i], factors[i], ranks[i], fdtype, outs[i], ALTO_VAR_GENERIC, osz,
                      fs[(dev_groups.size() + k) % branches]);
  }
  for (int k = 0; e == cudaSuccess && k < branches; ++k) {
    e = cudaEventRecord(join[k], fs[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join[k], 0);
  }
  if (e == cudaSuccess && !hot_items.empty()) {
    const int64_t tot = hot_prefix.back();
    int64_t gsz = (tot + 255) / 256;
    if (gsz > static_cast<int64_t>(sms) * 16) gsz = static_cast<int64_t>(sms) * 16;
    if (osz == 8)
      hot_reduce_batch_kernel<double><<<static_cast<unsigned>(gsz), 256, 0, s>>>(
          d_hot, d_hot_prefix, static_cast<int>(hot_items.size()));
    else
      hot_reduce_batch_kernel<float><<<static_cast<unsigned>(gsz), 256, 0, s>>>(
          d_hot, d_hot_prefix, static_cast<int>(hot_items.size()));
    note_launch();
    e = cudaGetLastError();
  }
  cudaGraph_t graph = nullptr;
  if (capturing) {
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = e2;
  }
  // kernels captured, not launched: counted at every alto_batch_run instead
  const int kernels = static_cast<int>(launch_total() - launches0);
  note_launch(-kernels);
  if (e == cudaSuccess) {
    b->graph = graph;
    e = cudaGraphInstantiate(&b->exec, graph, 0);
  } else if (graph) {
    cudaGraphDestroy(graph);
  }
  for (int k = 0; k < branches; ++k) {
    if (join[k]) cudaEventDestroy(join[k]);
    if (fs[k]) cudaStreamDestroy(fs[k]);
  }
  if (fork) cudaEventDestroy(fork);
  if (own) cudaStreamDestroy(own);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_plan(b);
    delete b;
    return fail(ALTO_ECUDA, "batch capture: %s", cudaGetErrorString(e));
  }
  b->groups = static_cast<int>(dev_groups.size());
  b->single = static_cast<int>(single.size());
  b->kernels = kernels;
  *out = b;
  return ALTO_OK;
}

alto_status alto_batch_run(alto_batch_t b, void* stream) {
  if (b == nullptr) return fail(ALTO_EINVAL, "null batch");
  const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(ALTO_ECUDA, "batch run: %s", cudaGetErrorString(e));
  note_launch(b->kernels);
  return ALTO_OK;
}

alto_status alto_batch_info(alto_batch_t b, int* items, int* groups, int* single, int* kernels) {
  if (b == nullptr) return fail(ALTO_EINVAL, "null batch");
  if (kernels) *kernels = b->kernels;
  if (items) *items = b->items;
  if (groups) *groups = b->groups;
  if (single) *single = b->single;
  return ALTO_OK;
}

alto_status alto_batch_destroy(alto_batch_t b) {
  if (b == nullptr) return ALTO_OK;
  free_plan(b);
  delete b;
  return ALTO_OK;
}

}  // extern "C"
