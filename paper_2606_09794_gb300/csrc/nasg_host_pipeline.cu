// Fused forward+backward for parameters and outputs in HOST memory
// (nasgabor_fused_fwd_bwd_host). Page-locked arrays are read and written in place
// by the kernel (register path) over the chip-to-chip link. Otherwise the
// primitives are processed in chunks that
// flow through three device slots, with the host->device copies of chunk i+1,
// the kernel of chunk i and the device->host copies of chunk i-1 in flight at
// the same time (two internal copy streams plus the caller's stream, ordered by
// events). On a Grace-Blackwell node the copies run over the chip-to-chip link
// in both directions at once, so a step costs about max(inputs in, outputs out)
// instead of their sum. Plane-major arrays move with one strided 2D copy per
// chunk (all planes of the chunk's span).
#include <mutex>

#include "nasg_kernels.cuh"

namespace nasg {
namespace {

constexpr int kSlots = 3;
constexpr int kMaxDevices = 64;

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct SlotLayout {
  size_t params, c0, means, g_rgb, rgb, g_params, g_c0, g_means, bytes;
};

inline SlotLayout slot_layout(int P, int L, int es, int64_t chunk) {
  SlotLayout s{};
  size_t o = 0;
  auto take = [&](size_t b) { const size_t at = o; o = al256(o + b); return at; };
  const size_t cl = size_t(chunk) * size_t(L);
  s.params = take(size_t(P) * cl * es);
  s.c0 = take(3 * size_t(chunk) * es);
  s.means = take(size_t(chunk) * 12);
  s.g_rgb = take(size_t(chunk) * 12);
  s.rgb = take(size_t(chunk) * 12);
  s.g_params = take(size_t(P) * cl * 4);
  s.g_c0 = take(3 * size_t(chunk) * 4);
  s.g_means = take(size_t(chunk) * 12);
  s.bytes = o;
  return s;
}

// Per device: two non-blocking copy streams and the ordering events of a call
// (timing disabled), created on first use and kept for the life of the process,
// and a lock that a call holds while it enqueues, so that calls from several host
// threads on one device take the copy streams and events in turn.
struct Pipeline {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, in_done[kSlots] = {}, k_done[kSlots] = {}, out_done[kSlots] = {};
  bool ready = false;
  std::mutex call;
};
Pipeline g_pipes[kMaxDevices];
std::mutex g_pipes_mu;

Pipeline* device_pipeline() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pipes_mu);
  Pipeline& p = g_pipes[dev];
  if (!p.ready) {
    auto ev = [](cudaEvent_t& e) { return e || cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess; };
    bool ok = (p.in || cudaStreamCreateWithFlags(&p.in, cudaStreamNonBlocking) == cudaSuccess) &&
              (p.out || cudaStreamCreateWithFlags(&p.out, cudaStreamNonBlocking) == cudaSuccess) && ev(p.start);
    for (int s = 0; ok && s < kSlots; ++s) ok = ev(p.in_done[s]) && ev(p.k_done[s]) && ev(p.out_done[s]);
    if (!ok) return nullptr;
    p.ready = true;
  }
  return &p;
}

// The device address of page-locked host memory at p (mapped into the device's
// address space), or nullptr for any other memory (pageable, device, unknown).
const void* mapped_host(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // an unregistered pointer is not an error of this call
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

}  // namespace
}  // namespace nasg

using namespace nasg;

extern "C" size_t nasgabor_fused_host_workspace_bytes(const nasg_desc* desc, int64_t chunk) {
  if (check_desc(desc) != NASG_OK || chunk < 8 || chunk % 8 != 0 || chunk > (int64_t(1) << 26)) return 0;
  const int P = nasg_param_planes(desc->frame_mode, desc->lobe_family);
  if (P < 0) return 0;
  return kSlots * slot_layout(P, desc->n_lobes, elem_size(desc->param_dtype), chunk).bytes;
}

extern "C" nasg_status nasgabor_fused_fwd_bwd_host(const nasg_desc* desc, const void* params, const void* c0,
                                                   const float* means, const float* cam, const float* g_rgb,
                                                   float* rgb, float* g_params, float* g_c0, float* g_means,
                                                   int64_t chunk, void* workspace, size_t workspace_bytes,
                                                   void* stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
  if (desc->accumulate != 0) return NASG_ERR_RANGE;
  if (chunk < 8 || chunk % 8 != 0 || chunk > (int64_t(1) << 26)) return NASG_ERR_RANGE;
  if (desc->n == 0) return NASG_OK;
  if (!params || !c0 || !means || !cam || !g_rgb || !rgb || !g_params || !g_c0 || !workspace) return NASG_ERR_NULL;
  if (!aligned(workspace, 256)) return NASG_ERR_ALIGN;
  const int P = nasg_param_planes(desc->frame_mode, desc->lobe_family);
  if (P < 0) return NASG_ERR_UNSUPPORTED;
  const int L = desc->n_lobes;
  const int es = elem_size(desc->param_dtype);
  const SlotLayout sl = slot_layout(P, L, es, chunk);
  if (workspace_bytes < kSlots * sl.bytes) return NASG_ERR_RANGE;
  {
    // Every array page-locked: the kernel reads and writes them in place over the
    // host link (plain loads and stores; no copies, no workspace).
    const void* hp[8] = {params, c0, means, g_rgb, rgb, g_params, g_c0, g_means};
    const void* dp[8] = {};
    bool direct = true;
    for (int j = 0; j < 8 && direct; ++j) direct = (j == 7 && !hp[j]) || (dp[j] = mapped_host(hp[j])) != nullptr;
    if (direct)
      return fused_fwd_bwd_register_path(desc, dp[0], dp[1], static_cast<const float*>(dp[2]), cam,
                                         static_cast<const float*>(dp[3]), static_cast<float*>(const_cast<void*>(dp[4])),
                                         static_cast<float*>(const_cast<void*>(dp[5])),
                                         static_cast<float*>(const_cast<void*>(dp[6])),
                                         static_cast<float*>(const_cast<void*>(dp[7])), as_stream(stream));
  }
  Pipeline* pipe = device_pipeline();
  if (!pipe) return check_launch();
  std::lock_guard<std::mutex> call_lock(pipe->call);
  Pipeline& cs = *pipe;
  cudaStream_t comp = as_stream(stream);
  const int64_t n = desc->n;
  const size_t NL = size_t(n) * L;
  const unsigned char* ph = static_cast<const unsigned char*>(params);
  const unsigned char* ch = static_cast<const unsigned char*>(c0);
  unsigned char* ws = static_cast<unsigned char*>(workspace);

  cudaEvent_t start = cs.start;
  cudaEvent_t* in_done = cs.in_done;
  cudaEvent_t* k_done = cs.k_done;
  cudaEvent_t* out_done = cs.out_done;
  // everything queued on the caller's stream so far happens first
  bool ok = cudaEventRecord(start, comp) == cudaSuccess && cudaStreamWaitEvent(cs.in, start, 0) == cudaSuccess &&
       cudaStreamWaitEvent(cs.out, start, 0) == cudaSuccess;
  const int64_t n_chunks = (n + chunk - 1) / chunk;
  for (int64_t i = 0; ok && st == NASG_OK && i < n_chunks; ++i) {
    const int s = int(i % kSlots);
    unsigned char* base = ws + size_t(s) * sl.bytes;
    const int64_t i0 = i * chunk;
    const int64_t cnt = (n - i0 < chunk) ? n - i0 : chunk;
    const size_t cl = size_t(cnt) * L;
    // inputs: wait until the kernel of the slot's previous chunk has read them
    if (i >= kSlots) ok = ok && cudaStreamWaitEvent(cs.in, k_done[s], 0) == cudaSuccess;
    ok = ok && cudaMemcpy2DAsync(base + sl.params, cl * es, ph + size_t(i0) * L * es, NL * es, cl * es, P,
                                 cudaMemcpyHostToDevice, cs.in) == cudaSuccess;
    ok = ok && cudaMemcpy2DAsync(base + sl.c0, size_t(cnt) * es, ch + size_t(i0) * es, size_t(n) * es,
                                 size_t(cnt) * es, 3, cudaMemcpyHostToDevice, cs.in) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(base + sl.means, means + 3 * i0, size_t(cnt) * 12, cudaMemcpyHostToDevice,
                               cs.in) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(base + sl.g_rgb, g_rgb + 3 * i0, size_t(cnt) * 12, cudaMemcpyHostToDevice,
                               cs.in) == cudaSuccess;
    ok = ok && cudaEventRecord(in_done[s], cs.in) == cudaSuccess;
    // kernel: after its inputs landed and the slot's previous outputs left
    ok = ok && cudaStreamWaitEvent(comp, in_done[s], 0) == cudaSuccess;
    if (i >= kSlots) ok = ok && cudaStreamWaitEvent(comp, out_done[s], 0) == cudaSuccess;
    if (!ok) break;
    nasg_desc d = *desc;
    d.n = cnt;
    st = nasgabor_fused_fwd_bwd(&d, base + sl.params, base + sl.c0, reinterpret_cast<const float*>(base + sl.means),
                                cam, reinterpret_cast<const float*>(base + sl.g_rgb),
                                reinterpret_cast<float*>(base + sl.rgb), reinterpret_cast<float*>(base + sl.g_params),
                                reinterpret_cast<float*>(base + sl.g_c0),
                                g_means ? reinterpret_cast<float*>(base + sl.g_means) : nullptr, comp);
    ok = ok && cudaEventRecord(k_done[s], comp) == cudaSuccess;
    // outputs
    ok = ok && cudaStreamWaitEvent(cs.out, k_done[s], 0) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(rgb + 3 * i0, base + sl.rgb, size_t(cnt) * 12, cudaMemcpyDeviceToHost, cs.out) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy2DAsync(reinterpret_cast<unsigned char*>(g_params) + size_t(i0) * L * 4, NL * 4,
                                 base + sl.g_params, cl * 4, cl * 4, P, cudaMemcpyDeviceToHost, cs.out) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy2DAsync(reinterpret_cast<unsigned char*>(g_c0) + size_t(i0) * 4, size_t(n) * 4,
                                 base + sl.g_c0, size_t(cnt) * 4, size_t(cnt) * 4, 3, cudaMemcpyDeviceToHost,
                                 cs.out) == cudaSuccess;
    if (g_means)
      ok = ok && cudaMemcpyAsync(g_means + 3 * i0, base + sl.g_means, size_t(cnt) * 12, cudaMemcpyDeviceToHost,
                                 cs.out) == cudaSuccess;
    ok = ok && cudaEventRecord(out_done[s], cs.out) == cudaSuccess;
  }
  // the caller's stream resumes after the last outputs are back in host memory
  if (ok) ok = cudaEventRecord(start, cs.out) == cudaSuccess && cudaStreamWaitEvent(comp, start, 0) == cudaSuccess;
  if (st != NASG_OK) return st;
  return ok ? NASG_OK : check_launch();
}
