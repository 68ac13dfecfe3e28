// C ABI of libvqd (declared in include/vqd.h): contexts, argument checks, launch accounting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <functional>
#include <memory>
#include <thread>
#include <string>
#include <vector>

#include "fused.h"
#include "kernels.h"
#include "tcgemm.h"
#include "vqd_internal.h"

using namespace vqd;

namespace {

thread_local std::string g_err;

struct KClass {
  const char* name;
};
enum StatClass { SC_ELEM, SC_SUP1, SC_UNI2, SC_SUP2, SC_FUSED, SC_BATCH, SC_REDUCE, SC_INIT, SC_TC_COMPOSE, SC_TC_GEMM,
                 SC_COUNT };
const char* kStatNames[SC_COUNT] = {"elem",   "sup1", "uni2",       "sup2",   "fused_stage",
                                    "batch",  "reduce", "init", "tc_compose", "tc_gemm"};

struct Stat {
  int64_t launches = 0;
  double ms = 0, bytes = 0, amp_updates = 0, fma = 0;
};

void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  cudaGetLastError();  // clear a sticky-free error so later calls can report their own
  throw Error(e == cudaErrorMemoryAllocation ? VQD_ENOMEM : VQD_EDEVICE,
              std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

struct vqd_ctx {
  int prec = VQD_F64;
  size_t esize = 16;
  std::vector<int> n;
  std::vector<size_t> off;  // byte offset of each instance
  char* base = nullptr;
  bool owns = false;
  size_t total = 0;
  cudaStream_t stream = nullptr;
  double* d_scratch = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;
  std::string err;
  unsigned flags = 0;
  // launch accounting
  int prof = 0;
  Stat stats[SC_COUNT];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evpool;
  std::vector<int> pending;  // class of the launch timed by evpool[i]
  FusedCache fused;          // device buffers of the fused path
  // Batched path: its own device buffers, and the CUDA graph of the last batch (replayed when the
  // same program runs again on a capturable stream).
  FusedCache batch;
  uint64_t batch_key = 0;
  cudaGraphExec_t batch_graph = nullptr;
  std::vector<int> batch_passes;
  std::vector<double> batch_traffic;  // state sizes read and written per instance (1 + frac per stage)
  std::vector<size_t> batch_nops;
  int64_t batch_waves = 0;
  TileShape shape;           // tile shape of the fused and batched paths (defaults per precision)
  // Tensor-core path: second state buffer (out-of-place GEMMs), composition buffer, tiled limbs, error flag.
  void* tc_alt = nullptr;
  size_t tc_alt_cap = 0;
  void* tc_S = nullptr;
  size_t tc_S_cap = 0;
  void* tc_R = nullptr;
  size_t tc_R_cap = 0;
  int* tc_err = nullptr;

  char* ptr(int inst) { return base + off[inst]; }
  size_t bytes(int inst) const { return vqd_state_bytes(n[inst], prec); }
};

static void set_err(vqd_ctx* c, const std::string& m) {
  if (c) c->err = m;
  g_err = m;
}

#define API_BEGIN try {
#define API_END(ctx)                                   \
  }                                                    \
  catch (const Error& e) {                             \
    set_err(ctx, e.what());                            \
    return e.code;                                     \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    set_err(ctx, "host allocation failed");            \
    return VQD_ENOMEM;                                 \
  }                                                    \
  catch (const std::exception& e) {                    \
    set_err(ctx, e.what());                            \
    return VQD_EINVAL;                                 \
  }                                                    \
  return VQD_OK;

static void harvest(vqd_ctx* c) {
  if (c->pending.empty()) return;
  cuda_check(cudaStreamSynchronize(c->stream), "synchronise for timing");
  for (size_t i = 0; i < c->pending.size(); i++) {
    float ms = 0;
    cuda_check(cudaEventElapsedTime(&ms, c->evpool[i].first, c->evpool[i].second), "event timing");
    c->stats[c->pending[i]].ms += ms;
  }
  c->pending.clear();
}

// Run `launch` (which enqueues kernels on c->stream) with launch accounting for class `cls`.
template <class F>
static void timed(vqd_ctx* c, int cls, double bytes, double amp_updates, int64_t launches, F&& launch) {
  if (c->prof == 2) {
    if (c->pending.size() >= 4096) harvest(c);
    size_t i = c->pending.size();
    if (i >= c->evpool.size()) {
      cudaEvent_t a, b;
      cuda_check(cudaEventCreate(&a), "event create");
      cuda_check(cudaEventCreate(&b), "event create");
      c->evpool.emplace_back(a, b);
    }
    cuda_check(cudaEventRecord(c->evpool[i].first, c->stream), "event record");
    cuda_check(launch(), kStatNames[cls]);
    cuda_check(cudaEventRecord(c->evpool[i].second, c->stream), "event record");
    c->pending.push_back(cls);
  } else {
    cuda_check(launch(), kStatNames[cls]);
  }
  if (c->prof) {
    Stat& s = c->stats[cls];
    s.launches += launches;
    s.bytes += bytes;
    s.amp_updates += amp_updates;
  }
}

static vqd_ctx* need_ctx(vqd_t c) {
  if (!c) throw Error(VQD_EINVAL, "NULL context");
  return c;
}
static void need_inst(vqd_ctx* c, int inst) {
  if (inst < 0 || inst >= (int)c->n.size()) throw Error(VQD_EINVAL, "instance index out of range");
}
static void need_targets(vqd_ctx* c, int inst, int k, const int* t) {
  if (k < 1 || k > 2) throw Error(VQD_EINVAL, "k must be 1 or 2");
  if (!t) throw Error(VQD_EINVAL, "NULL targets");
  for (int j = 0; j < k; j++) {
    if (t[j] < 0 || t[j] >= c->n[inst]) throw Error(VQD_EINVAL, "target qubit out of range");
    for (int i = 0; i < j; i++)
      if (t[i] == t[j]) throw Error(VQD_EINVAL, "repeated target qubit");
  }
}

static void apply_op(vqd_ctx* c, int inst, const Op& op) {
  Pass p = classify(op);
  const int n = c->n[inst];
  static const int cls_of[4] = {SC_ELEM, SC_SUP1, SC_UNI2, SC_SUP2};
  timed(c, cls_of[p.kind], 2.0 * c->bytes(inst) * pass_touched_fraction(p), op.weight * std::ldexp(1.0, 2 * n), 1,
        [&] { return launch_pass(c->prec, c->ptr(inst), n, p, c->stream); });
  if (c->prof) c->stats[cls_of[p.kind]].fma += pass_fma_per_amp(p, c->prec != VQD_F32) * std::ldexp(1.0, 2 * n);
}

static std::vector<cd> to_cd(const vqd_c128* m, size_t cnt) {
  std::vector<cd> v(cnt);
  for (size_t i = 0; i < cnt; i++) v[i] = cd(m[i].re, m[i].im);
  return v;
}

static void alloc_aux(vqd_ctx* c) {
  cuda_check(cudaMalloc(&c->d_scratch, sizeof(double) * reduce_scratch_doubles()), "scratch allocation");
  cuda_check(cudaMalloc(&c->d_out, sizeof(double) * reduce_out_doubles()), "result allocation");
  cuda_check(cudaMallocHost(&c->h_out, sizeof(double) * reduce_out_doubles()), "pinned result allocation");
}

static void free_ctx(vqd_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& e : c->evpool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  fused_cache_free(c->fused);
  if (c->batch_graph) cudaGraphExecDestroy(c->batch_graph);
  fused_cache_free(c->batch);
  for (void* q : {c->tc_alt, c->tc_S, c->tc_R, (void*)c->tc_err})
    if (q) cudaFree(q);
  if (c->owns && c->base) cudaFree(c->base);
  if (c->d_scratch) cudaFree(c->d_scratch);
  if (c->d_out) cudaFree(c->d_out);
  if (c->h_out) cudaFreeHost(c->h_out);
  delete c;
}

static vqd_ctx* make_ctx(int count, const int* n, int prec, void* stream, void* dev, size_t dev_bytes) {
  if (prec != VQD_F64 && prec != VQD_F32 && prec != VQD_F32_SPLIT)
    throw Error(VQD_EINVAL, "precision must be VQD_F64, VQD_F32 or VQD_F32_SPLIT");
  if (count < 1) throw Error(VQD_EINVAL, "count must be >= 1");
  std::unique_ptr<vqd_ctx, void (*)(vqd_ctx*)> c(new vqd_ctx, free_ctx);
  c->prec = prec;
  c->esize = prec == VQD_F32 ? 8 : 16;
  c->stream = (cudaStream_t)stream;
  size_t total = 0;
  for (int i = 0; i < count; i++) {
    if (n[i] < 1 || n[i] > VQD_MAX_QUBITS) throw Error(VQD_EINVAL, "qubit count outside 1..16");
    c->n.push_back(n[i]);
    c->off.push_back(total);
    total += (vqd_state_bytes(n[i], prec) + 255) / 256 * 256;
  }
  c->total = total;
  if (dev) {
    if (dev_bytes < vqd_state_bytes(n[0], prec)) throw Error(VQD_EINVAL, "device buffer too small");
    if ((uintptr_t)dev % 16) throw Error(VQD_EINVAL, "device buffer must be 16-byte aligned");
    c->base = (char*)dev;
    c->owns = false;
  } else {
    cuda_check(cudaMalloc(&c->base, total), "state allocation");
    c->owns = true;
  }
  alloc_aux(c.get());
  return c.release();
}

namespace vqd {
int report_static_error(int code, const char* msg) {
  set_err(nullptr, msg);
  return code;
}
}  // namespace vqd

using F_LAUNCH = std::function<cudaError_t()>;

// ================================================================== exported API
extern "C" {

size_t vqd_state_bytes(int n, int prec) {
  if (n < 1 || n > VQD_MAX_QUBITS) return 0;
  return (size_t)(prec == VQD_F32 ? 8 : 16) << (2 * n);
}

int vqd_create(int n, int prec, void* stream, vqd_t* out) {
  vqd_ctx* c = nullptr;
  API_BEGIN
  if (!out) throw Error(VQD_EINVAL, "NULL output handle");
  *out = nullptr;
  c = make_ctx(1, &n, prec, stream, nullptr, 0);
  cuda_check(launch_init_classical(c->prec, c->ptr(0), n, 0, c->stream), "init");
  *out = c;
  API_END(nullptr)
}

int vqd_create_batch(int count, const int* n, int prec, void* stream, vqd_t* out) {
  API_BEGIN
  if (!out || !n) throw Error(VQD_EINVAL, "NULL argument");
  *out = nullptr;
  vqd_ctx* c = make_ctx(count, n, prec, stream, nullptr, 0);
  for (int i = 0; i < count; i++) cuda_check(launch_init_classical(c->prec, c->ptr(i), n[i], 0, c->stream), "init");
  *out = c;
  API_END(nullptr)
}

int vqd_create_on(int n, int prec, void* dev_state, size_t bytes, void* stream, vqd_t* out) {
  API_BEGIN
  if (!out || !dev_state) throw Error(VQD_EINVAL, "NULL argument");
  *out = nullptr;
  *out = make_ctx(1, &n, prec, stream, dev_state, bytes);
  API_END(nullptr)
}

void vqd_destroy(vqd_t c) { free_ctx(c); }

int vqd_num_instances(vqd_t c) { return c ? (int)c->n.size() : VQD_EINVAL; }
int vqd_num_qubits(vqd_t c, int inst) {
  if (!c || inst < 0 || inst >= (int)c->n.size()) return VQD_EINVAL;
  return c->n[inst];
}
void* vqd_state_ptr(vqd_t c, int inst) {
  if (!c || inst < 0 || inst >= (int)c->n.size()) return nullptr;
  return c->ptr(inst);
}

int vqd_sync(vqd_t c) {
  API_BEGIN
  need_ctx(c);
  cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  API_END(c)
}

const char* vqd_last_error(vqd_t c) { return c ? c->err.c_str() : g_err.c_str(); }

int vqd_set_tile_shape(vqd_t c, int tile_bits, int passenger_bits) {
  API_BEGIN
  need_ctx(c);
  const int maxb = tile_bits_budget(c->prec);
  const int tb = tile_bits > 0 ? tile_bits : maxb;
  const int L = passenger_bits >= 0 ? passenger_bits : default_passengers(c->prec);
  if (tb > maxb || L > 3 || tb < 4 + L)
    throw Error(VQD_EINVAL, "tile shape: need 4 + passengers <= tile bits <= " + std::to_string(maxb) + ", passengers <= 3");
  c->shape.tile_bits = tile_bits;
  c->shape.passengers = passenger_bits;
  API_END(c)
}

int vqd_set_flags(vqd_t c, unsigned flags) {
  API_BEGIN
  need_ctx(c)->flags = flags;
  API_END(c)
}

int vqd_init_zero(vqd_t c, int inst) { return vqd_init_classical(c, inst, 0); }

int vqd_init_classical(vqd_t c, int inst, uint64_t basis) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (basis >= (1ull << c->n[inst])) throw Error(VQD_EINVAL, "basis state out of range");
  timed(c, SC_INIT, (double)c->bytes(inst), 0, 1,
        [&] { return launch_init_classical(c->prec, c->ptr(inst), c->n[inst], basis, c->stream); });
  API_END(c)
}

int vqd_init_product_diag(vqd_t c, int inst, const double* e) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (!e) throw Error(VQD_EINVAL, "NULL populations");
  for (int q = 0; q < c->n[inst]; q++)
    if (!(e[q] >= 0 && e[q] <= 1)) throw Error(VQD_EINVAL, "excited population outside [0,1]");
  timed(c, SC_INIT, (double)c->bytes(inst), 0, 1,
        [&] { return launch_init_product_diag(c->prec, c->ptr(inst), c->n[inst], e, c->stream); });
  API_END(c)
}

int vqd_apply_unitary(vqd_t c, int inst, int k, const int* t, const vqd_c128* U) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  need_targets(c, inst, k, t);
  if (!U) throw Error(VQD_EINVAL, "NULL matrix");
  Op op;
  op.unitary = true;
  op.k = k;
  for (int j = 0; j < k; j++) op.q[j] = t[j];
  op.m = to_cd(U, (size_t)1 << (2 * k));
  if (!(c->flags & VQD_NO_CHECK)) check_unitary(k, op.m.data());
  apply_op(c, inst, op);
  API_END(c)
}

int vqd_apply_kraus(vqd_t c, int inst, int k, const int* t, int nK, const vqd_c128* K) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  need_targets(c, inst, k, t);
  if (!K || nK < 1 || nK > 1024) throw Error(VQD_EINVAL, "need 1..1024 Kraus operators");
  std::vector<cd> ks = to_cd(K, (size_t)nK << (2 * k));
  if (!(c->flags & VQD_NO_CHECK)) check_cptn(k, nK, ks.data());
  Op op;
  op.unitary = false;
  op.k = k;
  for (int j = 0; j < k; j++) op.q[j] = t[j];
  op.m = superop_from_kraus(k, nK, ks.data());
  apply_op(c, inst, op);
  API_END(c)
}

int vqd_apply_superop(vqd_t c, int inst, int k, const int* t, const vqd_c128* S) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  need_targets(c, inst, k, t);
  if (!S) throw Error(VQD_EINVAL, "NULL matrix");
  Op op;
  op.unitary = false;
  op.k = k;
  for (int j = 0; j < k; j++) op.q[j] = t[j];
  op.m = to_cd(S, (size_t)1 << (4 * k));
  apply_op(c, inst, op);
  API_END(c)
}

static std::vector<Op> compile_list(vqd_ctx* c, int inst, int nops, const vqd_native_op* ops, unsigned flags) {
  if (nops < 0 || (nops > 0 && !ops)) throw Error(VQD_EINVAL, "bad op list");
  std::vector<Op> out;
  out.reserve(nops);
  for (int i = 0; i < nops; i++) {
    int ar = native_arity(ops[i].code);
    if (ar < 1) throw Error(VQD_EINVAL, "unknown native op code at index " + std::to_string(i));
    need_targets(c, inst, ar, ops[i].q);
    out.push_back(compile_native(ops[i], flags));
  }
  return out;
}

int vqd_apply_native(vqd_t c, int inst, int nops, const vqd_native_op* ops, unsigned flags) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  std::vector<Op> list = compile_list(c, inst, nops, ops, flags);
  for (const Op& op : list) apply_op(c, inst, op);
  API_END(c)
}

int vqd_run_program(vqd_t c, int inst, int nops, const vqd_native_op* ops, int fuse_qubits, unsigned flags) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  std::vector<Op> list = compile_list(c, inst, nops, ops, flags);
  const int n = c->n[inst];
  FusedPlan plan = plan_fused(list, n, c->prec, fuse_qubits, c->shape, (flags & VQD_HERMITIAN) != 0);
  upload_plan(c->fused, plan, c->prec, c->stream);
  for (size_t s = 0; s < plan.stages.size(); s++) {
    // a stage reads the tiles it runs (a fraction frac of the state) and writes the whole state
    const StageDesc& sd = plan.stages[s];
    timed(c, SC_FUSED, (1.0 + sd.frac) * c->bytes(inst), sd.weight * std::ldexp(1.0, 2 * n), 1,
          [&] { return launch_stage(c->fused, plan, (int)s, c->prec, c->ptr(inst), n, c->stream); });
    if (c->prof) c->stats[SC_FUSED].fma += sd.fma_per_amp * sd.frac * std::ldexp(1.0, 2 * n);
  }
  API_END(c)
}

// FNV-1a over the bytes of the batch description: identical programs give identical keys.
static uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

int vqd_run_batch(vqd_t c, const int64_t* offsets, const vqd_native_op* ops, int fuse_qubits, unsigned flags) {
  API_BEGIN
  need_ctx(c);
  if (!offsets || (offsets[c->n.size()] > 0 && !ops)) throw Error(VQD_EINVAL, "NULL offsets or ops");
  const int count = (int)c->n.size();
  for (int i = 0; i < count; i++)
    if (offsets[i] < 0 || offsets[i + 1] < offsets[i]) throw Error(VQD_EINVAL, "offsets must be non-decreasing");
  uint64_t key = 1469598103934665603ull;
  key = fnv1a(key, offsets, sizeof(int64_t) * (count + 1));
  key = fnv1a(key, ops, sizeof(vqd_native_op) * (size_t)offsets[count]);
  const int params[4] = {fuse_qubits, (int)flags, c->shape.tile_bits, c->shape.passengers};
  key = fnv1a(key, params, sizeof(params));
  auto account = [&](int64_t launches, F_LAUNCH launch) {
    double bytes = 0, upd = 0;
    for (int i = 0; i < count; i++) {
      bytes += c->bytes(i) * c->batch_traffic[i];
      upd += (double)c->batch_nops[i] * std::ldexp(1.0, 2 * c->n[i]);
    }
    timed(c, SC_BATCH, bytes, upd, launches, launch);
  };
  if (c->batch_graph && key == c->batch_key) {  // same batch as last time: replay its graph
    account(1, [&] { return cudaGraphLaunch(c->batch_graph, c->stream); });
    return VQD_OK;
  }
  // Instances are compiled and planned independently, on several host threads.
  std::vector<FusedPlan> plans(count);
  std::vector<size_t> nops(count);
  std::vector<std::string> errs(count);
  std::vector<int> codes(count, VQD_OK);
  const int nt = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int i = next++; i < count; i = next++) {
      try {
        std::vector<Op> list = compile_list(c, i, (int)(offsets[i + 1] - offsets[i]), ops + offsets[i], flags);
        nops[i] = list.size();
        plans[i] = plan_fused(list, c->n[i], c->prec, fuse_qubits, c->shape, (flags & VQD_HERMITIAN) != 0);
      } catch (const Error& e) {
        codes[i] = e.code;
        errs[i] = e.what();
      } catch (const std::exception& e) {
        codes[i] = VQD_EINVAL;
        errs[i] = e.what();
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; t++) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  for (int i = 0; i < count; i++)
    if (codes[i] != VQD_OK) throw Error(codes[i], "instance " + std::to_string(i) + ": " + errs[i]);
  BatchPlan plan = merge_batch(plans, c->n, c->off, c->prec);
  if (c->batch_graph) {
    cudaGraphExecDestroy(c->batch_graph);
    c->batch_graph = nullptr;
  }
  upload_batch(c->batch, plan, c->prec, c->stream);
  c->batch_passes = plan.passes;
  c->batch_traffic.assign(count, 0.0);
  for (int i = 0; i < count; i++)
    for (const StageDesc& sd : plans[i].stages) c->batch_traffic[i] += 1.0 + sd.frac;
  c->batch_nops = nops;
  c->batch_waves = (int64_t)plan.wave_begin.size() - 1;
  // On a stream that can be captured (not the legacy default stream), the waves are captured into
  // one CUDA graph, launched now and replayed by later calls with the same batch.
  if (c->stream != nullptr) {
    cudaGraph_t g = nullptr;
    cuda_check(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin graph capture");
    cudaError_t le = launch_batch(c->batch, plan, c->prec, c->base, c->stream);
    cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
    cuda_check(le, "batched waves (capture)");
    cuda_check(ce, "end graph capture");
    cudaError_t ie = cudaGraphInstantiate(&c->batch_graph, g, 0);
    cudaGraphDestroy(g);
    cuda_check(ie, "instantiate batch graph");
    c->batch_key = key;
    account(1, [&] { return cudaGraphLaunch(c->batch_graph, c->stream); });
  } else {
    account(c->batch_waves, [&] { return launch_batch(c->batch, plan, c->prec, c->base, c->stream); });
  }
  API_END(c)
}

// ---------------------------------------------------------------- tensor-core form of the fused path
static void grow_dev(void** p, size_t* cap, size_t need, const char* what) {
  if (need <= *cap) return;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cuda_check(cudaMalloc(p, need), what);
  *cap = need;
}

// Compile a native list for an n-qubit program without a context (host-only planning calls).
static std::vector<Op> compile_for(int n, int nops, const vqd_native_op* ops, unsigned flags) {
  if (n < 1 || n > VQD_MAX_QUBITS || nops < 0 || (nops > 0 && !ops)) throw Error(VQD_EINVAL, "bad argument");
  std::vector<Op> list;
  list.reserve(nops);
  for (int i = 0; i < nops; i++) {
    int ar = native_arity(ops[i].code);
    if (ar < 1) throw Error(VQD_EINVAL, "unknown native op code");
    for (int j = 0; j < ar; j++)
      if (ops[i].q[j] < 0 || ops[i].q[j] >= n || (j == 1 && ops[i].q[1] == ops[i].q[0]))
        throw Error(VQD_EINVAL, "bad target qubit");
    list.push_back(compile_native(ops[i], flags));
  }
  return list;
}

int vqd_tc_plan_info(int n, int nops, const vqd_native_op* ops, int k, unsigned flags, int64_t* info) {
  API_BEGIN
  if (!info) throw Error(VQD_EINVAL, "NULL info");
  if (k < 4 || k > 6 || k > n) throw Error(VQD_EINVAL, "k must be 4, 5 or 6 and at most n");
  std::vector<Op> list = compile_for(n, nops, ops, flags);
  std::vector<TcBlock> blocks = plan_tc_blocks(list, n, k);
  info[0] = (int64_t)blocks.size();
  info[1] = nops;
  info[2] = 0;
  for (const TcBlock& b : blocks) info[2] = std::max<int64_t>(info[2], (int64_t)b.ops.size());
  API_END(nullptr)
}

int vqd_run_program_tc(vqd_t c, int inst, int nops, const vqd_native_op* ops, int k, int scheme, unsigned flags) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (c->prec != VQD_F32) throw Error(VQD_ENOTSUP, "the tensor-core path needs a complex64 (VQD_F32) context");
  const int n = c->n[inst];
  if (k < 4 || k > 6 || k > n) throw Error(VQD_EINVAL, "k must be 4, 5 or 6 and at most the qubit count");
  if (scheme != VQD_TC_3XTF32 && scheme != VQD_TC_BF16X3) throw Error(VQD_EINVAL, "scheme must be VQD_TC_3XTF32 or VQD_TC_BF16X3");
  std::vector<Op> list = compile_list(c, inst, nops, ops, flags);
  std::vector<TcBlock> blocks = plan_tc_blocks(list, n, k);
  const size_t bytes = c->bytes(inst);
  grow_dev(&c->tc_alt, &c->tc_alt_cap, bytes, "tensor-core second state buffer");
  grow_dev(&c->tc_S, &c->tc_S_cap, tc_compose_bytes(k), "tensor-core composition buffer");
  grow_dev(&c->tc_R, &c->tc_R_cap, tc_r_bytes(k, scheme), "tensor-core operand limbs");
  if (!c->tc_err) cuda_check(cudaMalloc((void**)&c->tc_err, sizeof(int)), "tensor-core error flag");
  cuda_check(cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream), "clear error flag");
  char* cur = c->ptr(inst);
  char* other = (char*)c->tc_alt;
  for (const TcBlock& b : blocks) {
    // the block's qubits, ascending, padded with unused qubits up to k
    int q[6], nq = 0;
    for (int x = 0; x < n && nq < k; x++)
      if (b.qmask >> x & 1) q[nq++] = x;
    for (int x = 0; x < n && nq < k; x++)
      if (!(b.qmask >> x & 1)) q[nq++] = x;
    std::sort(q, q + k);
    int local[VQD_MAX_QUBITS];
    for (int j = 0; j < k; j++) local[q[j]] = j;
    // FP64 composition: the block's operators applied in order to the identity superoperator, as passes
    // of the plain FP64 kernels over the 2k-qubit composition layout
    timed(c, SC_TC_COMPOSE, 0.0, 0.0, (int64_t)b.ops.size() + 2, [&] {
      cudaError_t e = tc_compose_init(c->tc_S, k, c->stream);
      for (size_t i = 0; i < b.ops.size() && e == cudaSuccess; i++) {
        Op o = list[b.ops[i]];
        for (int j = 0; j < o.k; j++) o.q[j] = local[o.q[j]];
        e = launch_pass(VQD_F64, c->tc_S, 2 * k, classify(o), c->stream);
      }
      if (e == cudaSuccess) e = tc_build_r(c->tc_S, k, scheme, c->tc_R, c->stream);
      return e;
    });
    timed(c, SC_TC_GEMM, 2.0 * (double)bytes, b.weight * std::ldexp(1.0, 2 * n), 1,
          [&] { return tc_apply(cur, other, n, k, q, scheme, c->tc_R, c->tc_err, c->stream); });
    std::swap(cur, other);
  }
  if (cur != c->ptr(inst))
    cuda_check(cudaMemcpyAsync(c->ptr(inst), cur, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy back");
  int herr = 0;
  cuda_check(cudaMemcpyAsync(&herr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error flag");
  cuda_check(cudaStreamSynchronize(c->stream), "tensor-core path");
  if (herr) throw Error(VQD_EDEVICE, "tensor-core kernel: a bounded wait expired (copy or tensor-core operation did not complete)");
  API_END(c)
}

int vqd_compile_op(const vqd_native_op* op, unsigned flags, int* is_unitary, int* k, int* targets, vqd_c128* mat) {
  API_BEGIN
  if (!op || !is_unitary || !k || !targets || !mat) throw Error(VQD_EINVAL, "NULL argument");
  Op o = compile_native(*op, flags);
  *is_unitary = o.unitary ? 1 : 0;
  *k = o.k;
  for (int j = 0; j < o.k; j++) targets[j] = o.q[j];
  for (size_t i = 0; i < o.m.size(); i++) mat[i] = {o.m[i].real(), o.m[i].imag()};
  API_END(nullptr)
}

int vqd_plan_info(int n, int prec, int nops, const vqd_native_op* ops, int fuse_qubits, int tile_bits,
                  int passenger_bits, unsigned flags, int64_t* info) {
  API_BEGIN
  if (!info || n < 1 || n > VQD_MAX_QUBITS || nops < 0 || (nops > 0 && !ops)) throw Error(VQD_EINVAL, "bad argument");
  if (prec != VQD_F64 && prec != VQD_F32 && prec != VQD_F32_SPLIT) throw Error(VQD_EINVAL, "bad precision");
  std::vector<Op> list;
  list.reserve(nops);
  for (int i = 0; i < nops; i++) {
    int ar = native_arity(ops[i].code);
    if (ar < 1) throw Error(VQD_EINVAL, "unknown native op code");
    for (int j = 0; j < ar; j++)
      if (ops[i].q[j] < 0 || ops[i].q[j] >= n || (j == 1 && ops[i].q[1] == ops[i].q[0]))
        throw Error(VQD_EINVAL, "bad target qubit");
    list.push_back(compile_native(ops[i], flags));
  }
  TileShape shape;
  shape.tile_bits = tile_bits;
  shape.passengers = passenger_bits;
  FusedPlan plan = plan_fused(list, n, prec, fuse_qubits, shape, (flags & VQD_HERMITIAN) != 0);
  for (int i = 0; i < 8; i++) info[i] = 0;
  info[0] = (int64_t)plan.stages.size();
  info[1] = (int64_t)plan.blocks.size();
  for (const BlockOp& t : plan.ops) {
    const int cls = (t.kind == BK_DIAG_A || t.kind == BK_DIAG_B || t.kind == BK_DIAG2) ? 0
                    : (t.kind == BK_SUP1_A || t.kind == BK_SUP1_B)                     ? 1
                    : t.kind == BK_UNI2                                                ? 2
                                                                                       : 3;
    info[2 + cls] += 1;
  }
  info[6] = plan.max_bits;
  info[7] = nops;
  API_END(nullptr)
}

int vqd_schedule(int n, int nin, const vqd_native_op* in, const double* dur, int idle_code, const double* t1,
                 const double* t2, int cap, vqd_native_op* out, int* nout) {
  API_BEGIN
  if (n < 1 || n > 32 || nin < 0 || (nin > 0 && (!in || !dur)) || !t1 || !t2 || !out || !nout || cap < 0)
    throw Error(VQD_EINVAL, "bad argument");
  if (idle_code != VQD_OP_IDLE && idle_code != VQD_OP_IDLE_DEPOL && idle_code != VQD_OP_IDLE_T2S)
    throw Error(VQD_EINVAL, "idle_code must be an idle op");
  // gates with their trailing noise ops, each assigned to a layer
  struct G {
    int first, count;  // gate op and its noise ops: in[first .. first+count)
    int layer;
  };
  std::vector<G> gates;
  std::vector<int> ready(n, 0);  // first layer qubit j is free in
  for (int i = 0; i < nin; i++) {
    const int ar = native_arity(in[i].code);
    if (ar < 1 || in[i].nq != ar) throw Error(VQD_EINVAL, "bad native op at index " + std::to_string(i));
    for (int j = 0; j < ar; j++)
      if (in[i].q[j] < 0 || in[i].q[j] >= n) throw Error(VQD_EINVAL, "qubit out of range at index " + std::to_string(i));
    if (dur[i] < 0) {
      if (gates.empty() || gates.back().first + gates.back().count != i)
        throw Error(VQD_EINVAL, "noise op at index " + std::to_string(i) + " does not follow a gate");
      gates.back().count++;
      continue;
    }
    int layer = 0;
    for (int j = 0; j < ar; j++) layer = std::max(layer, ready[in[i].q[j]]);
    for (int j = 0; j < ar; j++) ready[in[i].q[j]] = layer + 1;
    gates.push_back({i, 1, layer});
  }
  int nl = 0;
  for (const G& g : gates) nl = std::max(nl, g.layer + 1);
  int cnt = 0;
  auto emit = [&](const vqd_native_op& o) {
    if (cnt >= cap) throw Error(VQD_EINVAL, "output capacity too small");
    out[cnt++] = o;
  };
  for (int l = 0; l < nl; l++) {
    double len = 0;
    std::vector<double> busy(n, 0.0);
    for (const G& g : gates) {
      if (g.layer != l) continue;
      const double d = dur[g.first];
      len = std::max(len, d);
      for (int j = 0; j < in[g.first].nq; j++) busy[in[g.first].q[j]] = d;
      for (int k = 0; k < g.count; k++) emit(in[g.first + k]);
    }
    for (int j = 0; j < n; j++) {
      const double dt = len - busy[j];
      if (dt <= 0) continue;
      vqd_native_op o;
      std::memset(&o, 0, sizeof(o));
      o.code = idle_code;
      o.nq = 1;
      o.q[0] = j;
      o.par[0] = dt;
      o.par[1] = t1[j];
      o.par[2] = t2[j];
      emit(o);
    }
  }
  *nout = cnt;
  API_END(nullptr)
}

// Output of the device compilers: counts every op and, when out is given, stores it (VQD_EINVAL once
// cap is exceeded).
struct OpSink {
  vqd_native_op* out;
  int cap;
  int cnt = 0;
  void put(const vqd_native_op& o) {
    if (out) {
      if (cnt >= cap) throw Error(VQD_EINVAL, "output capacity too small");
      out[cnt] = o;
    }
    cnt++;
  }
  void emit(int code, int q0, int q1, double p0, double p1 = 0, double p2 = 0, double p3 = 0) {
    vqd_native_op o;
    std::memset(&o, 0, sizeof(o));
    o.code = code;
    o.nq = q1 < 0 ? 1 : 2;
    o.q[0] = q0;
    o.q[1] = q1 < 0 ? 0 : q1;
    o.par[0] = p0; o.par[1] = p1; o.par[2] = p2; o.par[3] = p3;
    put(o);
  }
  // App. C: the error severities of a parameterised gate scale with its angle, eps -> eps |theta| / pi.
  // The standard error deph(p) o depol(q) of the gate's fidelity (App. B) becomes depol(q s) then
  // deph(p s); zero severities are left out.
  void scaled_stderr(int nq, int a, int b, double fbar, double x, double theta) {
    double pd, qd;
    stderr_params(nq, fbar, x, &pd, &qd);
    const double sc = std::fabs(theta) / 3.14159265358979323846;
    if (qd * sc > 0) emit(nq == 1 ? VQD_OP_DEPOL1 : VQD_OP_DEPOL2, a, nq == 1 ? -1 : b, qd * sc);
    if (pd * sc > 0) emit(nq == 1 ? VQD_OP_DEPH1 : VQD_OP_DEPH2, a, nq == 1 ? -1 : b, pd * sc);
  }
};

// Superconducting device compiler, Sec. 8 and the superconducting table of App. C: gates are exact
// and run in parallel (ASAP layers); the errors are the passive T1/T2 decay (gamp towards the thermal
// state, then the dephasing of Eq. depht2) of qubits outside an active gate, the static ZZ of every
// capacitively coupled pair not under a siZZle gate, and the readout's gamp(t_M) then depol(1 - F).
int vqd_sc_compile(const vqd_sc_device* dev, int nin, const vqd_native_op* in, int readout, int cap,
                   vqd_native_op* out, int* nout) {
  API_BEGIN
  if (!dev || !nout || nin < 0 || (nin > 0 && !in) || (out && cap < 0)) throw Error(VQD_EINVAL, "bad argument");
  const int n = dev->n;
  if (n < 1 || n > 32 || dev->ncouple < 0 || (dev->ncouple > 0 && (!dev->couple || !dev->coupling)))
    throw Error(VQD_EINVAL, "bad device: qubit count or coupling list");
  if (!dev->t1 || !dev->t2 || !dev->excited || !dev->freq || !dev->anharm) throw Error(VQD_EINVAL, "bad device: NULL table");
  for (int j = 0; j < n; j++) {
    if (!(dev->t1[j] > 0) || !(dev->t2[j] > 0)) throw Error(VQD_EINVAL, "bad device: T1 and T2 must be positive");
    if (!(dev->excited[j] >= 0 && dev->excited[j] <= 1)) throw Error(VQD_EINVAL, "bad device: excited population outside [0,1]");
    if (dev->fid_read && !(dev->fid_read[j] >= 0.25 && dev->fid_read[j] <= 1))
      throw Error(VQD_EINVAL, "bad device: readout fidelity outside [1/4,1]");
  }
  for (int k = 0; k < dev->ncouple; k++) {
    const int a = dev->couple[2 * k], b = dev->couple[2 * k + 1];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) throw Error(VQD_EINVAL, "bad device: coupled pair");
  }
  if (!(dev->dur_rxy >= 0 && dev->dur_zx >= 0 && dev->dur_zz >= 0 && dev->dur_meas >= 0))
    throw Error(VQD_EINVAL, "bad device: negative duration");
  const bool passive = !(dev->flags & VQD_SC_NO_PASSIVE), static_zz = !(dev->flags & VQD_SC_NO_STATIC_ZZ);
  // layer of every gate (a gate starts once all its qubits are free), and its duration
  std::vector<int> layer(nin), ready(n, 0);
  std::vector<double> dur(nin);
  int nl = 0;
  for (int i = 0; i < nin; i++) {
    const vqd_native_op& o = in[i];
    switch (o.code) {
      case VQD_OP_RX: case VQD_OP_RY: dur[i] = dev->dur_rxy; break;
      case VQD_OP_RZ: dur[i] = 0; break;  // virtual Z (Sec. 8)
      case VQD_OP_ZX: dur[i] = dev->dur_zx; break;
      case VQD_OP_ZZ: dur[i] = dev->dur_zz; break;
      default: throw Error(VQD_EINVAL, "op " + std::to_string(i) + " is not a superconducting native gate");
    }
    const int ar = native_arity(o.code);
    if (o.nq != ar) throw Error(VQD_EINVAL, "bad arity at op " + std::to_string(i));
    int l = 0;
    for (int j = 0; j < ar; j++) {
      if (o.q[j] < 0 || o.q[j] >= n || (j == 1 && o.q[1] == o.q[0]))
        throw Error(VQD_EINVAL, "bad qubit at op " + std::to_string(i));
      l = std::max(l, ready[o.q[j]]);
    }
    for (int j = 0; j < ar; j++) ready[o.q[j]] = l + 1;
    layer[i] = l;
    nl = std::max(nl, l + 1);
  }
  std::vector<std::vector<int>> by_layer(nl);
  for (int i = 0; i < nin; i++) by_layer[layer[i]].push_back(i);
  OpSink sink{out, cap};
  const double two_pi = 2 * 3.14159265358979323846;
  auto decay = [&](int j, double dt) {  // free-induction decay of qubit j over dt
    sink.emit(VQD_OP_GAMP, j, -1, dt, dev->t1[j], 1 - dev->excited[j], 0);
    sink.emit(VQD_OP_DEPH1, j, -1, 0.5 * (1 - std::exp(-dt / dev->t2[j])), 0, 0, 0);
  };
  for (int l = 0; l < nl; l++) {
    double len = 0;
    std::vector<double> busy(n, 0.0);
    for (int i : by_layer[l]) {
      sink.put(in[i]);
      len = std::max(len, dur[i]);
      for (int j = 0; j < in[i].nq; j++) busy[in[i].q[j]] = dur[i];
    }
    if (len <= 0) continue;
    if (static_zz) {
      for (int k = 0; k < dev->ncouple; k++) {
        const int c = dev->couple[2 * k], t = dev->couple[2 * k + 1];
        bool sizzle = false;  // a siZZle gate on the pair replaces its static ZZ (Sec. 8)
        for (int i : by_layer[l])
          if (in[i].code == VQD_OP_ZZ && ((in[i].q[0] == c && in[i].q[1] == t) || (in[i].q[0] == t && in[i].q[1] == c)))
            sizzle = true;
        if (sizzle || dev->coupling[k] == 0) continue;
        // frequencies (MHz) times the layer length (us) as angles: beta is then the accumulated phase
        const double w = two_pi * len;
        sink.emit(VQD_OP_ZZ_STATIC, c, t, w * dev->coupling[k], w * (dev->freq[c] - dev->freq[t]), w * dev->anharm[t],
             w * dev->anharm[c]);
      }
    }
    if (passive)
      for (int j = 0; j < n; j++)
        if (len - busy[j] > 0) decay(j, len - busy[j]);
  }
  if (readout)
    for (int j = 0; j < n; j++) {
      if (passive && dev->dur_meas > 0) sink.emit(VQD_OP_GAMP, j, -1, dev->dur_meas, dev->t1[j], 1 - dev->excited[j], 0);
      if (dev->fid_read) sink.emit(VQD_OP_DEPOL1, j, -1, 1 - dev->fid_read[j], 0, 0, 0);
    }
  *nout = sink.cnt;
  API_END(nullptr)
}

// Silicon spin device compiler, Sec. 7 and the silicon table of App. C: gates run one at a time.
// Rx/Ry: the standard error of Sec. 3.2 from the single-qubit fidelity, the off-resonant drive of
// Eq. (off_resonant) on every other qubit, passive T1/T2 decay (Eqs. depolt1, depht2) of the other
// qubits, and the off-state conditional-Rz crosstalk on the pairs of passive neighbours.  CZ/CPh on a
// neighbour pair: its standard error, the on-state crosstalk controlled-Rz(delta theta / pi) on every
// other neighbour pair, and the passive decay.  Rz is virtual: no time, no noise.
int vqd_si_compile(const vqd_si_device* dev, int nin, const vqd_native_op* in, int cap, vqd_native_op* out,
                   int* nout) {
  API_BEGIN
  if (!dev || !nout || nin < 0 || (nin > 0 && !in) || (out && cap < 0)) throw Error(VQD_EINVAL, "bad argument");
  const int n = dev->n;
  if (n < 2 || n > 32) throw Error(VQD_EINVAL, "bad device: qubit count");
  if (!dev->t1 || !dev->t2 || !dev->freq || !dev->rabi || !dev->fid_1q || !dev->freq_cz || !dev->fid_cz)
    throw Error(VQD_EINVAL, "bad device: NULL table");
  for (int j = 0; j < n; j++)
    if (!(dev->t1[j] > 0) || !(dev->t2[j] > 0) || !(dev->rabi[j] > 0) || !(dev->fid_1q[j] > 0 && dev->fid_1q[j] <= 1))
      throw Error(VQD_EINVAL, "bad device: T1, T2, Rabi frequency or fidelity");
  for (int k = 0; k + 1 < n; k++)
    if (!(dev->freq_cz[k] > 0) || !(dev->fid_cz[k] > 0 && dev->fid_cz[k] <= 1))
      throw Error(VQD_EINVAL, "bad device: CZ frequency or fidelity");
  if (!(dev->x_1q >= 0 && dev->x_1q <= 1 && dev->x_cz >= 0 && dev->x_cz <= 1))
    throw Error(VQD_EINVAL, "bad device: depolarising fraction outside [0,1]");
  const bool passive = !(dev->flags & VQD_SI_NO_PASSIVE), offres = !(dev->flags & VQD_SI_NO_OFFRES);
  const double two_pi = 2 * 3.14159265358979323846;
  OpSink sink{out, cap};
  auto decay_others = [&](int a, int b, double t) {  // passive qubits over the gate's duration
    if (!passive || t <= 0) return;
    for (int j = 0; j < n; j++)
      if (j != a && j != b) sink.emit(VQD_OP_IDLE_DEPOL, j, -1, t, dev->t1[j], dev->t2[j]);
  };
  for (int i = 0; i < nin; i++) {
    const vqd_native_op& o = in[i];
    const int ar = native_arity(o.code);
    if (ar < 1 || o.nq != ar) throw Error(VQD_EINVAL, "bad op at index " + std::to_string(i));
    for (int j = 0; j < ar; j++)
      if (o.q[j] < 0 || o.q[j] >= n || (j == 1 && o.q[1] == o.q[0]))
        throw Error(VQD_EINVAL, "bad qubit at op " + std::to_string(i));
    if (o.code == VQD_OP_RZ) {  // virtual
      sink.put(o);
      continue;
    }
    if (o.code == VQD_OP_RX || o.code == VQD_OP_RY) {
      const int q = o.q[0];
      const double t = std::fabs(o.par[0]) / (two_pi * dev->rabi[q]);  // rotation angle 2 pi f_Rabi t
      sink.put(o);
      sink.scaled_stderr(1, q, -1, dev->fid_1q[q], dev->x_1q, o.par[0]);
      if (offres && t > 0)
        for (int j = 0; j < n; j++)
          if (j != q)
            sink.emit(VQD_OP_OFFRES, j, -1, two_pi * dev->rabi[q], two_pi * std::fabs(dev->freq[j] - dev->freq[q]), t);
      decay_others(q, -1, t);
      if (dev->xtalk_off)
        for (int k = 0; k + 1 < n; k++)
          if (k != q && k + 1 != q && dev->xtalk_off[k] != 0) sink.emit(VQD_OP_CRZ_XTALK, k, k + 1, dev->xtalk_off[k], 0, 0);
      continue;
    }
    if (o.code == VQD_OP_CZ || o.code == VQD_OP_CPH) {
      const int a = o.q[0], b = o.q[1];
      if (std::abs(a - b) != 1) throw Error(VQD_EINVAL, "controlled phase on non-neighbours at op " + std::to_string(i));
      const int k = std::min(a, b);
      const double theta = o.code == VQD_OP_CZ ? 3.14159265358979323846 : o.par[0];
      const double t = std::fabs(theta) / (two_pi * dev->freq_cz[k]);  // conditional phase 2 pi f_CZ t
      sink.put(o);
      sink.scaled_stderr(2, a, b, dev->fid_cz[k], dev->x_cz, theta);
      if (dev->xtalk_on)
        for (int j = 0; j + 1 < n; j++) {
          const double d = dev->xtalk_on[k * (n - 1) + j];
          if (j != k && d != 0) sink.emit(VQD_OP_CRZ_XTALK, j, j + 1, d * theta / 3.14159265358979323846, 0, 0);
        }
      decay_others(a, b, t);
      continue;
    }
    throw Error(VQD_EINVAL, "op " + std::to_string(i) + " is not a silicon native gate");
  }
  *nout = sink.cnt;
  API_END(nullptr)
}

// NV-centre device compiler, Sec. 5 and the NV-centre table of App. C: serial gates, each followed by
// its standard error (Sec. 3.2 with the table's depolarising:dephasing split); the qubits outside a gate
// feel the weak ZZ among nuclear spins and the passive T1/T2 decay (Eqs. depolt1, depht2) for its
// duration; the electron readout's bias is an amplitude damping between two X gates.
int vqd_nv_compile(const vqd_nv_device* dev, int nin, const vqd_native_op* in, int readout, int cap,
                   vqd_native_op* out, int* nout) {
  API_BEGIN
  if (!dev || !nout || nin < 0 || (nin > 0 && !in) || (out && cap < 0)) throw Error(VQD_EINVAL, "bad argument");
  const int n = dev->n;
  if (n < 2 || n > 32) throw Error(VQD_EINVAL, "bad device: qubit count");
  if (!dev->t1 || !dev->t2 || !dev->freq_xy || !dev->freq_z || !dev->fid_xy || !dev->fid_z || !dev->freq_crot ||
      !dev->fid_crot)
    throw Error(VQD_EINVAL, "bad device: NULL table");
  for (int j = 0; j < n; j++)
    if (!(dev->t1[j] > 0) || !(dev->t2[j] > 0) || !(dev->freq_xy[j] > 0) || !(dev->freq_z[j] > 0) ||
        !(dev->fid_xy[j] > 0 && dev->fid_xy[j] <= 1) || !(dev->fid_z[j] > 0 && dev->fid_z[j] <= 1))
      throw Error(VQD_EINVAL, "bad device: T1, T2, frequency or fidelity");
  for (int j = 0; j + 1 < n; j++)
    if (!(dev->freq_crot[j] > 0) || !(dev->fid_crot[j] > 0 && dev->fid_crot[j] <= 1))
      throw Error(VQD_EINVAL, "bad device: conditional-rotation frequency or fidelity");
  if (!(dev->x_xy >= 0 && dev->x_xy <= 1 && dev->x_crot >= 0 && dev->x_crot <= 1))
    throw Error(VQD_EINVAL, "bad device: depolarising fraction outside [0,1]");
  if (readout && !(dev->fid_meas >= 0 && dev->fid_meas <= 1 && dev->dur_meas >= 0))
    throw Error(VQD_EINVAL, "bad device: readout fidelity or duration");
  const bool passive = !(dev->flags & VQD_NV_NO_PASSIVE);
  const double two_pi = 2 * 3.14159265358979323846;
  OpSink sink{out, cap};
  auto passive_noise = [&](int a, int b, double t) {  // qubits outside the gate, for its duration
    if (!passive || t <= 0) return;
    if (dev->freq_zz != 0)
      for (int i = 1; i < n; i++)
        for (int k = i + 1; k < n; k++)
          if (i != a && i != b && k != a && k != b) sink.emit(VQD_OP_ZZ_IDLE, i, k, t, dev->freq_zz, 0);
    for (int j = 0; j < n; j++)
      if (j != a && j != b) sink.emit(VQD_OP_IDLE_DEPOL, j, -1, t, dev->t1[j], dev->t2[j]);
  };
  for (int i = 0; i < nin; i++) {
    const vqd_native_op& o = in[i];
    const int ar = native_arity(o.code);
    if (ar < 1 || o.nq != ar) throw Error(VQD_EINVAL, "bad op at index " + std::to_string(i));
    for (int j = 0; j < ar; j++)
      if (o.q[j] < 0 || o.q[j] >= n || (j == 1 && o.q[1] == o.q[0]))
        throw Error(VQD_EINVAL, "bad qubit at op " + std::to_string(i));
    if (o.code == VQD_OP_RX || o.code == VQD_OP_RY || o.code == VQD_OP_RZ) {
      const int q = o.q[0];
      const bool z = o.code == VQD_OP_RZ;
      const double t = std::fabs(o.par[0]) / (two_pi * (z ? dev->freq_z[q] : dev->freq_xy[q]));
      sink.put(o);
      if (!z) sink.scaled_stderr(1, q, -1, dev->fid_xy[q], dev->x_xy, o.par[0]);
      else if (dev->fid_z[q] < 1) sink.scaled_stderr(1, q, -1, dev->fid_z[q], 0.0, o.par[0]);
      passive_noise(q, -1, t);
      continue;
    }
    if (o.code == VQD_OP_ZX || o.code == VQD_OP_ZY) {
      if (o.q[0] != 0) throw Error(VQD_EINVAL, "conditional rotation not controlled by the electron (qubit 0) at op " +
                                                   std::to_string(i));
      const int j = o.q[1];
      const double t = std::fabs(o.par[0]) / (two_pi * dev->freq_crot[j - 1]);
      sink.put(o);
      sink.scaled_stderr(2, 0, j, dev->fid_crot[j - 1], dev->x_crot, o.par[0]);
      passive_noise(0, j, t);
      continue;
    }
    throw Error(VQD_EINVAL, "op " + std::to_string(i) + " is not an NV-centre native gate");
  }
  if (readout) {
    const double pi = 3.14159265358979323846;
    sink.emit(VQD_OP_RX, 0, -1, pi, 0, 0);
    sink.emit(VQD_OP_AMP, 0, -1, 1 - dev->fid_meas, 0, 0);
    sink.emit(VQD_OP_RX, 0, -1, pi, 0, 0);
    passive_noise(0, -1, dev->dur_meas);
  }
  *nout = sink.cnt;
  API_END(nullptr)
}

// Trapped-ion device compiler, Sec. 4 and the trapped-ion table of App. C (zones and shuttling left
// out): serial gates, each x/y rotation or CZ followed by its standard error (App. B, App. C's angle
// rule), passive T1 as depolarising and Gaussian T2* dephasing on the other ions, and readout as a
// symmetric bit flip per ion, one ion at a time.
int vqd_ion_compile(const vqd_ion_device* dev, int nin, const vqd_native_op* in, int readout, int cap,
                    vqd_native_op* out, int* nout) {
  API_BEGIN
  if (!dev || !nout || nin < 0 || (nin > 0 && !in) || (out && cap < 0)) throw Error(VQD_EINVAL, "bad argument");
  const int n = dev->n;
  if (n < 1 || n > 32) throw Error(VQD_EINVAL, "bad device: ion count");
  if (!(dev->t1 > 0) || !(dev->t2s > 0) || !(dev->rabi > 0) || !(dev->freq_cz > 0))
    throw Error(VQD_EINVAL, "bad device: T1, T2*, Rabi or CZ frequency");
  if (!(dev->fid_xy > 0 && dev->fid_xy <= 1) || !(dev->fid_cz > 0 && dev->fid_cz <= 1) ||
      !(dev->x_xy >= 0 && dev->x_xy <= 1) || !(dev->x_cz >= 0 && dev->x_cz <= 1))
    throw Error(VQD_EINVAL, "bad device: fidelity or depolarising fraction");
  if (readout && !(dev->bf_read >= 0 && dev->bf_read <= 0.5 && dev->dur_read >= 0))
    throw Error(VQD_EINVAL, "bad device: readout bit flip or duration");
  const bool passive = !(dev->flags & VQD_ION_NO_PASSIVE);
  const double pi = 3.14159265358979323846;
  OpSink sink{out, cap};
  auto idle_others = [&](int a, int b, double t, int from) {  // ions from.. outside the gate, for t
    if (!passive || t <= 0) return;
    for (int j = from; j < n; j++)
      if (j != a && j != b) sink.emit(VQD_OP_IDLE_T2S, j, -1, t, dev->t1, dev->t2s);
  };
  for (int i = 0; i < nin; i++) {
    const vqd_native_op& o = in[i];
    const int ar = native_arity(o.code);
    if (ar < 1 || o.nq != ar) throw Error(VQD_EINVAL, "bad op at index " + std::to_string(i));
    for (int j = 0; j < ar; j++)
      if (o.q[j] < 0 || o.q[j] >= n || (j == 1 && o.q[1] == o.q[0]))
        throw Error(VQD_EINVAL, "bad qubit at op " + std::to_string(i));
    if (o.code == VQD_OP_RZ) {  // virtual: instantaneous and exact
      sink.put(o);
    } else if (o.code == VQD_OP_RX || o.code == VQD_OP_RY) {
      sink.put(o);
      sink.scaled_stderr(1, o.q[0], -1, dev->fid_xy, dev->x_xy, o.par[0]);
      idle_others(o.q[0], -1, std::fabs(o.par[0]) / (2 * pi * dev->rabi), 0);
    } else if (o.code == VQD_OP_CZ) {
      sink.put(o);
      sink.scaled_stderr(2, o.q[0], o.q[1], dev->fid_cz, dev->x_cz, pi);
      idle_others(o.q[0], o.q[1], 1.0 / (2 * dev->freq_cz), 0);
    } else {
      throw Error(VQD_EINVAL, "op " + std::to_string(i) + " is not a trapped-ion native gate");
    }
  }
  if (readout)
    for (int j = 0; j < n; j++) {
      if (dev->bf_read > 0) sink.emit(VQD_OP_BITFLIP, j, -1, dev->bf_read, 0, 0);
      idle_others(-1, -1, dev->dur_read, j + 1);
    }
  *nout = sink.cnt;
  API_END(nullptr)
}

// Neutral-atom device compiler, Sec. 6 and the neutral-atom table of App. C (static sites; moves, loss
// and multi-qubit gates left out): serial gates; a Raman rotation is followed by its phase error and the
// asymmetric bit flip, a Rydberg CZ by the leakage of Eq. czleak; the other atoms decay passively.
int vqd_na_compile(const vqd_na_device* dev, int nin, const vqd_native_op* in, int init, int readout, int cap,
                   vqd_native_op* out, int* nout) {
  API_BEGIN
  if (!dev || !nout || nin < 0 || (nin > 0 && !in) || (out && cap < 0)) throw Error(VQD_EINVAL, "bad argument");
  const int n = dev->n;
  if (n < 1 || n > 32 || !dev->x || !dev->y) throw Error(VQD_EINVAL, "bad device: atom count or sites");
  if (!(dev->t2 > 0) || !(dev->t_vac > 0) || !(dev->blockade >= 0) || !(dev->dur_cz >= 0))
    throw Error(VQD_EINVAL, "bad device: T2, vacuum lifetime, blockade radius or CZ duration");
  auto unit = [](double v) { return v >= 0 && v <= 1; };
  if (!unit(dev->p10) || !unit(dev->p01) || !unit(dev->leak_init) || !unit(dev->leak_cz_a) || !unit(dev->leak_cz_b))
    throw Error(VQD_EINVAL, "bad device: a probability outside [0,1]");
  if (readout && !(dev->fid_meas >= 0.5 && dev->fid_meas <= 1)) throw Error(VQD_EINVAL, "bad device: readout fidelity");
  const bool passive = !(dev->flags & VQD_NA_NO_PASSIVE);
  const double pi = 3.14159265358979323846, t1 = dev->t_vac / n;
  OpSink sink{out, cap};
  auto idle_others = [&](int a, int b, double t) {
    if (!passive || t <= 0) return;
    for (int j = 0; j < n; j++)
      if (j != a && j != b) sink.emit(VQD_OP_IDLE_DEPOL, j, -1, t, t1, dev->t2);
  };
  if (init)
    for (int j = 0; j < n; j++) sink.emit(VQD_OP_LEAK_INIT, j, -1, dev->leak_init);
  for (int i = 0; i < nin; i++) {
    const vqd_native_op& o = in[i];
    const int ar = native_arity(o.code);
    if (ar < 1 || o.nq != ar) throw Error(VQD_EINVAL, "bad op at index " + std::to_string(i));
    for (int j = 0; j < ar; j++)
      if (o.q[j] < 0 || o.q[j] >= n || (j == 1 && o.q[1] == o.q[0]))
        throw Error(VQD_EINVAL, "bad qubit at op " + std::to_string(i));
    if (o.code == VQD_OP_U) {
      const int q = o.q[0];
      const double t = std::fabs(o.par[3]);
      const double sc = std::hypot(o.par[1], o.par[2]) * t / pi;  // rotation angle over pi
      sink.put(o);
      sink.emit(VQD_OP_DEPH1, q, -1, 1 - std::exp(-t / (2 * dev->t2)));
      if ((dev->p10 > 0 || dev->p01 > 0) && sc > 0) sink.emit(VQD_OP_BITFLIP_ASYM, q, -1, dev->p10 * sc, dev->p01 * sc);
      idle_others(q, -1, t);
    } else if (o.code == VQD_OP_CZPHI) {
      const int a = o.q[0], b = o.q[1];
      if (std::hypot(dev->x[a] - dev->x[b], dev->y[a] - dev->y[b]) > dev->blockade)
        throw Error(VQD_EINVAL, "CZ(phi) on atoms farther apart than the blockade radius at op " + std::to_string(i));
      sink.put(o);
      sink.emit(VQD_OP_LEAK_CZ, a, b, dev->leak_cz_a, dev->leak_cz_b);
      idle_others(a, b, dev->dur_cz);
    } else {
      throw Error(VQD_EINVAL, "op " + std::to_string(i) + " is not a neutral-atom native gate");
    }
  }
  if (readout)
    for (int j = 0; j < n; j++) sink.emit(VQD_OP_DEPOL1, j, -1, 1.5 * (1 - dev->fid_meas));
  *nout = sink.cnt;
  API_END(nullptr)
}

int vqd_stderr_params(int nq, double fbar, double x, double* p, double* q) {
  API_BEGIN
  if (!p || !q) throw Error(VQD_EINVAL, "NULL output");
  stderr_params(nq, fbar, x, p, q);
  API_END(nullptr)
}

static void fetch(vqd_ctx* c, size_t cnt) {
  cuda_check(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream), "D2H result");
  cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
}

int vqd_prob(vqd_t c, int inst, int m, const int* qubits, double* out) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  const int n = c->n[inst];
  if (m < 1 || m > n || !qubits || !out) throw Error(VQD_EINVAL, "bad qubit list");
  unsigned used = 0;
  for (int j = 0; j < m; j++) {
    if (qubits[j] < 0 || qubits[j] >= n || (used >> qubits[j] & 1)) throw Error(VQD_EINVAL, "bad or repeated qubit");
    used |= 1u << qubits[j];
  }
  timed(c, SC_REDUCE, std::ldexp(1.0, n) * c->esize, 0, 2,
        [&] { return launch_prob(c->prec, c->ptr(inst), n, m, qubits, c->d_scratch, c->d_out, c->stream); });
  fetch(c, (size_t)1 << m);
  std::memcpy(out, c->h_out, sizeof(double) << m);
  API_END(c)
}

int vqd_batch_reduce(vqd_t c, double* probs, double* trace_re, double* purity) {
  API_BEGIN
  need_ctx(c);
  std::vector<unsigned char> items;
  std::vector<int> item_inst;
  batch_reduce_items(c->n, c->off, c->esize, items, item_inst);
  const size_t nitems = item_inst.size();
  size_t nprob = 0;
  for (int n : c->n) nprob += (size_t)1 << n;
  void *d_items = nullptr, *d_probs = nullptr, *d_part = nullptr;
  struct Free {
    void** p[3];
    ~Free() {
      for (void** q : p)
        if (*q) cudaFree(*q);
    }
  } guard{{&d_items, &d_probs, &d_part}};
  cuda_check(cudaMalloc(&d_items, items.size()), "batch reduce items");
  cuda_check(cudaMalloc(&d_probs, sizeof(double) * nprob), "batch reduce probabilities");
  cuda_check(cudaMalloc(&d_part, sizeof(double) * 3 * nitems), "batch reduce partials");
  cuda_check(cudaMemcpyAsync(d_items, items.data(), items.size(), cudaMemcpyHostToDevice, c->stream), "upload items");
  double bytes = 0;
  for (size_t i = 0; i < c->n.size(); i++) bytes += (double)c->bytes((int)i);
  timed(c, SC_REDUCE, bytes, 0, 1, [&] {
    return launch_batch_reduce(c->prec, c->base, c->n, c->off, (double*)d_probs, (double*)d_part, d_items, nitems,
                               c->stream);
  });
  std::vector<double> part(3 * nitems);
  cuda_check(cudaMemcpyAsync(part.data(), d_part, sizeof(double) * 3 * nitems, cudaMemcpyDeviceToHost, c->stream), "D2H");
  if (probs)
    cuda_check(cudaMemcpyAsync(probs, d_probs, sizeof(double) * nprob, cudaMemcpyDeviceToHost, c->stream), "D2H probs");
  cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  const size_t count = c->n.size();
  std::vector<double> tr(count, 0.0), pu(count, 0.0);
  for (size_t j = 0; j < nitems; j++) {  // chunks of one instance are summed in order
    tr[item_inst[j]] += part[3 * j];
    pu[item_inst[j]] += part[3 * j + 2];
  }
  for (size_t i = 0; i < count; i++) {
    if (trace_re) trace_re[i] = tr[i];
    if (purity) purity[i] = pu[i];
  }
  API_END(c)
}

int vqd_measure(vqd_t c, int inst, int q, double u, int force, int* outcome, double* prob) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  const int n = c->n[inst];
  if (q < 0 || q >= n) throw Error(VQD_EINVAL, "measured qubit out of range");
  if (force < -1 || force > 1) throw Error(VQD_EINVAL, "force must be -1 (draw), 0 or 1");
  if (force == -1 && !(u >= 0 && u < 1)) throw Error(VQD_EINVAL, "u must be in [0, 1)");
  timed(c, SC_REDUCE, std::ldexp(1.0, n) * c->esize, 0, 2,
        [&] { return launch_prob(c->prec, c->ptr(inst), n, 1, &q, c->d_scratch, c->d_out, c->stream); });
  fetch(c, 2);
  const double p0 = c->h_out[0], p1 = c->h_out[1], tot = p0 + p1;
  if (!(tot > 0)) throw Error(VQD_EINVAL, "state has zero trace");
  const int m = force >= 0 ? force : (u * tot < p0 ? 0 : 1);
  const double pm = m == 0 ? p0 : p1;
  if (!(pm > 0)) throw Error(VQD_EINVAL, "forced outcome has probability zero");
  // rho <- P_m rho P_m / tr(P_m rho): amplitudes whose row and column bit q both equal m are scaled,
  // all others vanish (a real diagonal superoperator on qubit q, member index r | c << 1)
  Pass p;
  p.kind = KK_ELEM;
  p.k = 1;
  p.q[0] = q;
  p.coef.assign(4, 0.0);
  p.coef[m | (m << 1)] = 1.0 / pm;
  timed(c, SC_ELEM, 2.0 * c->bytes(inst) * pass_touched_fraction(p), 0, 1,
        [&] { return launch_pass(c->prec, c->ptr(inst), n, p, c->stream); });
  if (outcome) *outcome = m;
  if (prob) *prob = pm / tot;
  API_END(c)
}

// Sec. 7, Eq. (m): projective parity measurement of (qa, qb), then optionally the decay map K of |01>
// into |10>.  Member index of the two-qubit block: r = a | b << 1 (a = qa's bit, b = qb's bit); the odd
// subspace is r in {1, 2}, the even one r in {0, 3}.
int vqd_measure_parity(vqd_t c, int inst, int qa, int qb, double u, int force, int decay, int* outcome,
                       double* prob) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  const int n = c->n[inst];
  if (qa < 0 || qa >= n || qb < 0 || qb >= n || qa == qb) throw Error(VQD_EINVAL, "measured qubits out of range or equal");
  if (force < -1 || force > 1) throw Error(VQD_EINVAL, "force must be -1 (draw), 0 or 1");
  if (force == -1 && !(u >= 0 && u < 1)) throw Error(VQD_EINVAL, "u must be in [0, 1)");
  const int qs[2] = {qa, qb};
  timed(c, SC_REDUCE, std::ldexp(1.0, n) * c->esize, 0, 2,
        [&] { return launch_prob(c->prec, c->ptr(inst), n, 2, qs, c->d_scratch, c->d_out, c->stream); });
  fetch(c, 4);
  const double podd = c->h_out[1] + c->h_out[2], peven = c->h_out[0] + c->h_out[3], tot = podd + peven;
  if (!(tot > 0)) throw Error(VQD_EINVAL, "state has zero trace");
  const int m = force >= 0 ? force : (u * tot < podd ? 0 : 1);
  const double pm = m == 0 ? podd : peven;
  if (!(pm > 0)) throw Error(VQD_EINVAL, "forced outcome has probability zero");
  auto in_sub = [&](int r) { return m == 0 ? (r == 1 || r == 2) : (r == 0 || r == 3); };
  Pass p;  // P_m rho P_m / p_m: a real diagonal superoperator, member s = r | c << 2
  p.kind = KK_ELEM;
  p.k = 2;
  p.q[0] = qa;
  p.q[1] = qb;
  p.coef.assign(16, 0.0);
  for (int s = 0; s < 16; s++)
    if (in_sub(s & 3) && in_sub(s >> 2)) p.coef[s] = 1.0 / pm;
  timed(c, SC_ELEM, 2.0 * c->bytes(inst) * pass_touched_fraction(p), 0, 1,
        [&] { return launch_pass(c->prec, c->ptr(inst), n, p, c->stream); });
  if (decay) {
    std::vector<cd> K(4 * 16, 0.0);  // row-major 4 x 4, index r = a | b << 1
    K[0 * 16 + 0 * 4 + 0] = 1.0;     // |00><00|
    K[1 * 16 + 3 * 4 + 3] = 1.0;     // |11><11|
    K[2 * 16 + 1 * 4 + 1] = 1.0;     // |10><10|  (a = 1, b = 0)
    K[3 * 16 + 1 * 4 + 2] = 1.0;     // |10><01|
    Op op;
    op.unitary = false;
    op.k = 2;
    op.q[0] = qa;
    op.q[1] = qb;
    op.m = superop_from_kraus(2, 4, K.data());
    op.weight = 0.0;
    apply_op(c, inst, op);
  }
  if (outcome) *outcome = m;
  if (prob) *prob = pm / tot;
  API_END(c)
}

int vqd_expect(vqd_t c, int inst, int nterms, const uint8_t* paulis, const double* coeffs, double* out) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (nterms < 0 || (nterms > 0 && (!paulis || !coeffs)) || !out) throw Error(VQD_EINVAL, "bad Pauli sum");
  const int n = c->n[inst];
  double total = 0;
  for (int t0 = 0; t0 < nterms; t0 += kExpectTermsPerLaunch) {
    int cnt = std::min(kExpectTermsPerLaunch, nterms - t0);
    std::vector<uint32_t> xm(cnt), zy(cnt);
    std::vector<int> ny(cnt);
    for (int t = 0; t < cnt; t++) {
      uint32_t x = 0, z = 0;
      int y = 0;
      for (int q = 0; q < n; q++) {
        uint8_t s = paulis[(size_t)(t0 + t) * n + q];
        if (s > 3) throw Error(VQD_EINVAL, "Pauli code must be 0..3");
        if (s == 1 || s == 2) x |= 1u << q;
        if (s == 2 || s == 3) z |= 1u << q;
        if (s == 2) y++;
      }
      xm[t] = x;
      zy[t] = z;
      ny[t] = y;
    }
    timed(c, SC_REDUCE, cnt * std::ldexp(1.0, n) * c->esize, 0, 3, [&] {
      return launch_expect(c->prec, c->ptr(inst), n, cnt, xm.data(), zy.data(), c->d_scratch, c->d_out, c->stream);
    });
    fetch(c, 2 * (size_t)cnt);
    // P|c> = i^{#Y} (-1)^{popc(c & zy)} |c ^ x>, so tr(P rho) = i^{#Y} sum_c (-1)^{...} rho[c][c ^ x]
    for (int t = 0; t < cnt; t++) {
      cd s(c->h_out[t], c->h_out[cnt + t]);
      static const cd ipow[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
      total += coeffs[t0 + t] * (ipow[ny[t] & 3] * s).real();
    }
  }
  *out = total;
  API_END(c)
}

int vqd_trace(vqd_t c, int inst, double* re, double* im) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (!re) throw Error(VQD_EINVAL, "NULL output");
  timed(c, SC_REDUCE, std::ldexp(1.0, c->n[inst]) * c->esize, 0, 2,
        [&] { return launch_trace(c->prec, c->ptr(inst), c->n[inst], c->d_scratch, c->d_out, c->stream); });
  fetch(c, 2);
  *re = c->h_out[0];
  if (im) *im = c->h_out[1];
  API_END(c)
}

int vqd_purity(vqd_t c, int inst, double* out) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (!out) throw Error(VQD_EINVAL, "NULL output");
  timed(c, SC_REDUCE, (double)c->bytes(inst), 0, 2,
        [&] { return launch_purity(c->prec, c->ptr(inst), c->n[inst], c->d_scratch, c->d_out, c->stream); });
  fetch(c, 1);
  *out = c->h_out[0];
  API_END(c)
}

int vqd_get_state(vqd_t c, int inst, vqd_c128* host) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (!host) throw Error(VQD_EINVAL, "NULL output");
  const size_t N = (size_t)1 << (2 * c->n[inst]);
  if (c->prec == VQD_F64) {
    cuda_check(cudaMemcpyAsync(host, c->ptr(inst), N * 16, cudaMemcpyDeviceToHost, c->stream), "D2H state");
    cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  } else if (c->prec == VQD_F32_SPLIT) {  // (re.hi, re.lo, im.hi, im.lo) -> hi + lo in FP64
    std::vector<float> tmp(4 * N);
    cuda_check(cudaMemcpyAsync(tmp.data(), c->ptr(inst), N * 16, cudaMemcpyDeviceToHost, c->stream), "D2H state");
    cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
    for (size_t i = 0; i < N; i++)
      host[i] = {(double)tmp[4 * i] + (double)tmp[4 * i + 1], (double)tmp[4 * i + 2] + (double)tmp[4 * i + 3]};
  } else {
    std::vector<float> tmp(2 * N);
    cuda_check(cudaMemcpyAsync(tmp.data(), c->ptr(inst), N * 8, cudaMemcpyDeviceToHost, c->stream), "D2H state");
    cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
    for (size_t i = 0; i < N; i++) host[i] = {tmp[2 * i], tmp[2 * i + 1]};
  }
  API_END(c)
}

int vqd_set_state(vqd_t c, int inst, const vqd_c128* host) {
  API_BEGIN
  need_ctx(c);
  need_inst(c, inst);
  if (!host) throw Error(VQD_EINVAL, "NULL input");
  const size_t N = (size_t)1 << (2 * c->n[inst]);
  if (c->prec == VQD_F64) {
    cuda_check(cudaMemcpyAsync(c->ptr(inst), host, N * 16, cudaMemcpyHostToDevice, c->stream), "H2D state");
    cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  } else if (c->prec == VQD_F32_SPLIT) {  // each double -> its nearest float and the float of the rest
    std::vector<float> tmp(4 * N);
    auto split = [](double d, float* w) {
      w[0] = (float)d;
      w[1] = (float)(d - (double)w[0]);
    };
    for (size_t i = 0; i < N; i++) {
      split(host[i].re, &tmp[4 * i]);
      split(host[i].im, &tmp[4 * i + 2]);
    }
    cuda_check(cudaMemcpyAsync(c->ptr(inst), tmp.data(), N * 16, cudaMemcpyHostToDevice, c->stream), "H2D state");
    cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  } else {
    std::vector<float> tmp(2 * N);
    for (size_t i = 0; i < N; i++) {
      tmp[2 * i] = (float)host[i].re;
      tmp[2 * i + 1] = (float)host[i].im;
    }
    cuda_check(cudaMemcpyAsync(c->ptr(inst), tmp.data(), N * 8, cudaMemcpyHostToDevice, c->stream), "H2D state");
    cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  }
  API_END(c)
}

int vqd_profile(vqd_t c, int mode) {
  API_BEGIN
  need_ctx(c);
  if (mode < 0 || mode > 2) throw Error(VQD_EINVAL, "mode must be 0, 1 or 2");
  harvest(c);
  c->prof = mode;
  API_END(c)
}

int vqd_profile_reset(vqd_t c) {
  API_BEGIN
  need_ctx(c);
  harvest(c);
  for (auto& s : c->stats) s = Stat();
  API_END(c)
}

int vqd_profile_read(vqd_t c, int max, vqd_kstat* out, int* n_out) {
  API_BEGIN
  need_ctx(c);
  if (!n_out || (max > 0 && !out)) throw Error(VQD_EINVAL, "NULL output");
  harvest(c);
  int cnt = 0;
  for (int i = 0; i < SC_COUNT; i++) {
    if (c->stats[i].launches == 0) continue;
    if (cnt < max) {
      vqd_kstat& k = out[cnt];
      std::memset(&k, 0, sizeof(k));
      std::strncpy(k.name, kStatNames[i], sizeof(k.name) - 1);
      k.launches = c->stats[i].launches;
      k.total_ms = c->stats[i].ms;
      k.alg_bytes = c->stats[i].bytes;
      k.amp_updates = c->stats[i].amp_updates;
      k.alg_fma = c->stats[i].fma;
    }
    cnt++;
  }
  *n_out = cnt;
  API_END(c)
}

}  // extern "C"
