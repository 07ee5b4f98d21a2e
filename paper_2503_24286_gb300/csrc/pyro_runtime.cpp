// libpyro C ABI: mechanism loading, NVRTC compilation with an on-disk cache,
// module management through driver entry points, argument checks, host-pointer
// staging and kernel launches.
#include "pyro.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "pyro_emit.h"
#include "pyro_emit_warp.h"
#include "pyro_internal.h"
#include "pyro_mech.h"

using namespace pyro;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

// ---- driver entry points (resolved through the runtime; no link to libcuda) ----
struct Driver {
  decltype(&cuModuleLoadData) ModuleLoadData = nullptr;
  decltype(&cuModuleUnload) ModuleUnload = nullptr;
  decltype(&cuModuleGetFunction) ModuleGetFunction = nullptr;
  decltype(&cuLaunchKernel) LaunchKernel = nullptr;
  decltype(&cuFuncSetAttribute) FuncSetAttribute = nullptr;
  decltype(&cuOccupancyMaxActiveBlocksPerMultiprocessor) Occupancy = nullptr;
  decltype(&cuOccupancyMaxActiveClusters) MaxActiveClusters = nullptr;
  decltype(&cuGetErrorString) GetErrorString = nullptr;
  bool ok = false;
  std::string err;
};

Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [&](const char* name, void** fn) {
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !*fn) {
        d.err = std::string("driver entry point ") + name + " unavailable: " + cudaGetErrorString(e);
        return false;
      }
      return true;
    };
    d.ok = get("cuModuleLoadData", (void**)&d.ModuleLoadData) &&
           get("cuModuleUnload", (void**)&d.ModuleUnload) &&
           get("cuModuleGetFunction", (void**)&d.ModuleGetFunction) &&
           get("cuLaunchKernel", (void**)&d.LaunchKernel) &&
           get("cuFuncSetAttribute", (void**)&d.FuncSetAttribute) &&
           get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void**)&d.Occupancy) &&
           get("cuOccupancyMaxActiveClusters", (void**)&d.MaxActiveClusters) &&
           get("cuGetErrorString", (void**)&d.GetErrorString);
  });
  return d;
}

std::string cu_err(CUresult r) {
  const char* s = nullptr;
  if (driver().GetErrorString) driver().GetErrorString(r, &s);
  return s ? s : ("CUresult " + std::to_string((int)r));
}

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char c : s) { h ^= c; h *= 1099511628211ull; }
  return h;
}

std::string cache_dir() {
  const char* d = std::getenv("PYRO_CACHE_DIR");
  if (d && *d) return d;
  const char* x = std::getenv("XDG_CACHE_HOME");
  std::string base = (x && *x) ? std::string(x) : std::string(std::getenv("HOME") ? std::getenv("HOME") : "/tmp") + "/.cache";
  return base + "/pyro_gb300";
}

void mkdirs(const std::string& path) {
  std::string cur;
  std::stringstream ss(path);
  std::string part;
  if (!path.empty() && path[0] == '/') cur = "/";
  while (std::getline(ss, part, '/')) {
    if (part.empty()) continue;
    cur += part + "/";
    mkdir(cur.c_str(), 0755);
  }
}

const char* kArch = "sm_103a";

// Compile CUDA C to a cubin for sm_103a with NVRTC.
bool nvrtc_compile(const std::string& src, std::vector<char>& cubin, std::string& log) {
  nvrtcProgram prog;
  const char* hdrs[] = {kDeviceMathSource};
  const char* names[] = {"pyro_device_math.cuh"};
  if (nvrtcCreateProgram(&prog, src.c_str(), "pyro_mech.cu", 1, hdrs, names) != NVRTC_SUCCESS) {
    log = "nvrtcCreateProgram failed";
    return false;
  }
  std::string arch = std::string("--gpu-architecture=") + kArch;
  // PYRO_NVRTC_VERBOSE=1: ptxas resource usage (registers, spills, shared memory) to stderr
  const bool verbose = std::getenv("PYRO_NVRTC_VERBOSE") != nullptr;
  const char* opts[] = {arch.c_str(), "-std=c++17", "-lineinfo", "-default-device", "--ptxas-options=-v"};
  nvrtcResult r = nvrtcCompileProgram(prog, verbose ? 5 : 4, opts);
  size_t ls = 0;
  nvrtcGetProgramLogSize(prog, &ls);
  log.assign(ls, '\0');
  if (ls) nvrtcGetProgramLog(prog, &log[0]);
  if (verbose) std::fprintf(stderr, "%s\n", log.c_str());
  if (r != NVRTC_SUCCESS) { nvrtcDestroyProgram(&prog); return false; }
  size_t cs = 0;
  nvrtcGetCUBINSize(prog, &cs);
  cubin.resize(cs);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return true;
}


// Compile CUDA C for sm_103a with NVRTC, or fetch the cubin from the on-disk
// cache keyed by a hash of the source, the device-math header, the arch and the
// NVRTC version.
int compile_cached(const std::string& src, bool use_cache, std::vector<char>& cubin) {
  if (const char* dump = std::getenv("PYRO_DUMP_DIR")) {   // debugging aid: keep the emitted sources
    mkdirs(dump);
    std::ofstream f(std::string(dump) + "/pyro_" + std::to_string(fnv1a(src) & 0xffffff) + ".cu");
    f << src;
  }
  int nv_major = 0, nv_minor = 0;
  nvrtcVersion(&nv_major, &nv_minor);
  std::string key_src = src + std::string(kDeviceMathSource) + kArch + std::to_string(nv_major) + "." +
                        std::to_string(nv_minor);
  char hex[32];
  std::snprintf(hex, sizeof hex, "%016llx", (unsigned long long)fnv1a(key_src));
  std::string dir = cache_dir(), path = dir + "/pyro_" + hex + ".cubin";
  cubin.clear();
  if (use_cache) {
    std::ifstream f(path, std::ios::binary);
    if (f) cubin.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
  }
  if (!cubin.empty()) return PYRO_OK;
  std::string log;
  if (!nvrtc_compile(src, cubin, log)) return fail(PYRO_ECOMPILE, "NVRTC: " + log);
  if (use_cache) {
    mkdirs(dir);
    std::string tmp = path + ".tmp" + std::to_string((long)getpid()) + "_" +
                      std::to_string((unsigned long long)std::hash<std::string>()(src) & 0xffff);
    std::ofstream f(tmp, std::ios::binary);
    f.write(cubin.data(), (std::streamsize)cubin.size());
    f.close();
    std::rename(tmp.c_str(), path.c_str());
  }
  return PYRO_OK;
}

struct Options {
  int block = 128;
  bool mixed = true;
  bool cache = true;
  bool checked = false;
  bool device = true;     // false: parse, validate, emit and compile only (no CUDA device needed)
  int deriv_block = 64;   // threads per block of the derivative kernels
  int store = 0;          // 0 auto, 1 shared memory, 2 global scratch (per-state species arrays)
  bool warp = false;      // net production rates: warp per state (table-driven) instead of thread per state
  int exp_ops = 4;        // exponential flavour (4 or 2 FP64 ops)
  int warp_exp_ops = 2;   // the warp-per-state kernels' exponential (compact code: 2 FP64 ops by default)
  bool exp_call = false;  // exponential as a called function
  bool cn_chord = false;  // Crank-Nicolson: keep a factorisation for several iterations (chord) instead of full Newton
  int cn_refresh = 4;     // chord: re-assemble and re-factor every cn_refresh-th iteration
  int jac_rows = 0;       // Jacobian row assembly: 0 auto (tables above 64 species), 1 inline, 2 tables
};

bool parse_options(const char* s, Options& o, std::string& err) {
  if (!s) return true;
  std::string str(s);
  for (char& c : str) if (c == ',') c = ';';
  std::stringstream ss(str);
  std::string kv;
  while (std::getline(ss, kv, ';')) {
    if (kv.empty()) continue;
    size_t eq = kv.find('=');
    if (eq == std::string::npos) { err = "option without '=': " + kv; return false; }
    std::string k = kv.substr(0, eq), v = kv.substr(eq + 1);
    if (k == "block") { o.block = std::atoi(v.c_str()); if (o.block < 32 || o.block > 512 || o.block % 32) { err = "block must be a multiple of 32 in [32, 512]"; return false; } }
    else if (k == "newton") { if (v == "mixed") o.mixed = true; else if (v == "fp64") o.mixed = false; else { err = "newton=mixed|fp64"; return false; } }
    else if (k == "cache") o.cache = v != "0";
    else if (k == "checked") o.checked = v != "0";
    else if (k == "device") o.device = v != "0";
    else if (k == "warp_exp") {
      if (v == "2") o.warp_exp_ops = 2;
      else if (v == "4") o.warp_exp_ops = 4;
      else { err = "warp_exp must be 2 or 4"; return false; }
    }
    else if (k == "exp") {
      if (v == "2") { o.exp_ops = 2; o.exp_call = false; }
      else if (v == "4") { o.exp_ops = 4; o.exp_call = false; }
      else if (v == "2call") { o.exp_ops = 2; o.exp_call = true; }
      else if (v == "4call") { o.exp_ops = 4; o.exp_call = true; }
      else { err = "exp=2|4|2call|4call"; return false; }
    }
    else if (k == "jac_rows") { if (v == "auto") o.jac_rows = 0; else if (v == "inline") o.jac_rows = 1; else if (v == "table") o.jac_rows = 2; else { err = "jac_rows=auto|inline|table"; return false; } }
    else if (k == "cn_refresh") { o.cn_refresh = std::atoi(v.c_str()); if (o.cn_refresh < 1 || o.cn_refresh > 1000) { err = "cn_refresh must be in [1, 1000]"; return false; } }
    else if (k == "cn_newton") { if (v == "full") o.cn_chord = false; else if (v == "chord") o.cn_chord = true; else { err = "cn_newton=full|chord"; return false; } }
    else if (k == "variant") { if (v == "thread") o.warp = false; else if (v == "warp") o.warp = true; else { err = "variant=thread|warp"; return false; } }
    else if (k == "store") { if (v == "auto") o.store = 0; else if (v == "shared") o.store = 1; else if (v == "global") o.store = 2; else { err = "store=auto|shared|global"; return false; } }
    else if (k == "deriv_block") { o.deriv_block = std::atoi(v.c_str()); if (o.deriv_block < 32 || o.deriv_block > 256 || o.deriv_block % 32) { err = "deriv_block must be a multiple of 32 in [32, 256]"; return false; } }
    else { err = "unknown option '" + k + "'"; return false; }
  }
  return true;
}

}  // namespace

struct pyro_mech {
  Mechanism m;
  Options opt;
  EmitResult emitted;
  std::vector<double> W;
  int device = -1;
  int num_sms = 0;
  CUmodule module = nullptr;
  CUfunction f_omega = nullptr, f_temperature = nullptr, f_energy = nullptr, f_density = nullptr,
             f_math = nullptr, f_enthalpy = nullptr, f_temperature_h = nullptr;
  int omega_blocks_per_sm = 1;
  unsigned long long* d_fail = nullptr;
  // derivative kernels: compiled and loaded on first use (or by pyro_mech_prepare)
  struct Group {
    CUmodule module = nullptr;
    CUfunction f = nullptr;
    int blocks_per_sm = 0;
    bool failed = false;
    std::string err;
    double* store = nullptr;   // per-block species arrays of this group (large mechanisms)
    std::map<std::string, CUfunction> fn;   // further kernels of the group
    int solve_blocks_per_sm = 0;            // Crank-Nicolson batched solve
    int residual_blocks_per_sm = 0;         // Crank-Nicolson right-hand side (chord iterations)
    int block = 0;                          // threads per block (0: the derivative block size)
    int smem = -1;                          // dynamic shared memory (-1: the derivative kernels')
    int clusters = 0;                       // clusters resident at once (clustered kernels)
  };
  std::map<std::string, Group> groups;
  std::mutex group_mu;
  double* d_jac_scratch = nullptr;
  size_t jac_scratch_bytes = 0;
  void* d_cn = nullptr;            // Crank-Nicolson per-chunk arrays (grows on demand)
  size_t cn_bytes = 0;
  double* d_store = nullptr;       // per-block species arrays when they do not fit in shared memory
  size_t store_bytes = 0;
  // learned initial guess
  pyro::MlpState* mlp = nullptr;
  float* mlp_norm_dev = nullptr;   // device copy of (e_mean, e_std, T_mean, T_std)
  CUfunction f_mlp_guess = nullptr, f_temperature_mlp = nullptr;
  // host-pointer calls: chunked copy-in / kernel / copy-out pipeline
  static constexpr int kSlots = 3;
  cudaStream_t pipe_stream[kSlots] = {};
  cudaEvent_t pipe_kdone[kSlots] = {};
  cudaEvent_t pipe_start = nullptr;
  std::vector<void*> stage[kSlots];
  std::vector<size_t> stage_bytes[kSlots];
  std::mutex mu;
};

namespace {

CUstream as_stream(void* s) { return (CUstream)s; }

// where a pointer lives: 1 device-accessible, 0 host, -1 invalid
int pointer_kind(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 1;
  return 0;
}

struct ArgSpec {
  const void* host;     // caller pointer (null: argument not used by this call)
  int64_t rows;         // the array is [rows][n], point index fastest
  size_t elem;          // bytes per element
  bool in, out;
};

// Classify the non-null pointers of a call: returns 1 (all device), 0 (all host) or -1 (mixed).
int classify(const std::vector<const void*>& ptrs) {
  int kind = -2;
  for (const void* p : ptrs) {
    if (!p) continue;
    int k = pointer_kind(p);
    if (kind == -2) kind = k;
    else if (kind != k) return -1;
  }
  return kind == -2 ? 1 : kind;
}

int ensure_stage(pyro_mech* h, int slot, size_t i, size_t bytes) {
  auto& buf = h->stage[slot];
  auto& have = h->stage_bytes[slot];
  if (buf.size() <= i) { buf.resize(i + 1, nullptr); have.resize(i + 1, 0); }
  if (have[i] < bytes) {
    if (buf[i]) cudaFree(buf[i]);
    buf[i] = nullptr;
    have[i] = 0;
    cudaError_t e = cudaMalloc(&buf[i], bytes);
    if (e != cudaSuccess) return fail(PYRO_ECUDA, std::string("staging allocation: ") + cudaGetErrorString(e));
    have[i] = bytes;
  }
  return PYRO_OK;
}

int ensure_pipe(pyro_mech* h) {
  if (h->pipe_start) return PYRO_OK;
  for (int s = 0; s < pyro_mech::kSlots; ++s) {
    if (cudaStreamCreateWithFlags(&h->pipe_stream[s], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->pipe_kdone[s], cudaEventDisableTiming) != cudaSuccess)
      return fail(PYRO_ECUDA, "creating the copy pipeline streams");
  }
  if (cudaEventCreateWithFlags(&h->pipe_start, cudaEventDisableTiming) != cudaSuccess)
    return fail(PYRO_ECUDA, "creating the copy pipeline streams");
  return PYRO_OK;
}

// `rows` rows of `width` bytes between pitched arrays: one 2D copy, or one copy
// per row where a pitch exceeds what a 2D copy accepts (2^31 - 1 bytes).
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, int64_t rows,
                      cudaMemcpyKind kind, cudaStream_t st) {
  if (rows == 1) return cudaMemcpyAsync(dst, src, width, kind, st);
  const size_t max_pitch = 2147483647u;
  if (dpitch <= max_pitch && spitch <= max_pitch)
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, (size_t)rows, kind, st);
  for (int64_t r = 0; r < rows; ++r) {
    cudaError_t e = cudaMemcpyAsync((char*)dst + r * dpitch, (const char*)src + r * spitch, width, kind, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Points per chunk of a host-pointer call: about 8 chunks, each large enough to
// fill the GPU, each slot's staging at most 1 GiB.
int64_t chunk_points(int64_t n, size_t bytes_per_point) {
  int64_t m = std::max<int64_t>((n + 7) / 8, 65536);
  int64_t cap = std::max<int64_t>(4096, (int64_t)(((size_t)1 << 30) / std::max<size_t>(bytes_per_point, 1)));
  m = std::min(m, cap);
  m = (m + 255) / 256 * 256;
  return std::min(m, n);
}

// Chunk sizes of a host-pointer call, each at most m points (one staging slot).
// Large calls ramp up from m/8 at the start and down to m/8 at the end: nothing
// overlaps the first copy-in and the last copy-out, so those stay short.
std::vector<int64_t> chunk_plan(int64_t n, int64_t m) {
  std::vector<int64_t> ramp, plan;
  if (m >= 8 * 256)
    for (int64_t a = m / 8; a < m; a *= 2) ramp.push_back((a + 255) / 256 * 256);
  int64_t ends = 0;
  for (int64_t a : ramp) ends += 2 * a;
  if (ramp.empty() || n < ends + m) {
    for (int64_t p = 0; p < n; p += m) plan.push_back(std::min(m, n - p));
    return plan;
  }
  for (int64_t a : ramp) plan.push_back(a);
  const int64_t mid = n - ends;
  for (int64_t p = 0; p < mid; p += m) plan.push_back(std::min(m, mid - p));
  for (auto it = ramp.rbegin(); it != ramp.rend(); ++it) plan.push_back(*it);
  return plan;
}

// Run `launch(device pointers, points, stream)` over n points.  Device pointers:
// one launch on the caller's stream.  Host pointers: chunks of points go through
// kSlots staging slots, each with its own stream, so that the copy-in of chunk
// c+1 and the copy-out of chunk c-1 overlap the kernel of chunk c.  Kernels that
// keep per-block scratch in global memory run one after another (event chain);
// with `concurrent` (no such scratch) the kernel of chunk c+1 may start while
// chunk c's last blocks still run.  A chunk of a [rows][n] array is a pitched 2D
// copy into a dense [rows][m] staging array, so the kernel sees the chunk as a
// problem of m points.  The call returns after the last copy-out has completed.
template <class F>
int with_args(pyro_mech* h, int64_t n, std::vector<ArgSpec> args, void* stream, F launch, bool concurrent = false) {
  std::vector<const void*> ptrs;
  for (auto& a : args) ptrs.push_back(a.host);
  int kind = classify(ptrs);
  if (kind < 0) return fail(PYRO_EINVAL, "arrays must be all device pointers or all host pointers");
  std::vector<void*> dev(args.size(), nullptr);
  if (kind == 1) {
    for (size_t i = 0; i < args.size(); ++i) dev[i] = const_cast<void*>(args[i].host);
    return launch(dev, n, stream);
  }
  std::lock_guard<std::mutex> lock(h->mu);
  if (int rc = ensure_pipe(h)) return rc;
  size_t per_point = 0;
  for (auto& a : args) if (a.host) per_point += (size_t)a.rows * a.elem;
  const int64_t m = chunk_points(n, per_point);
  const std::vector<int64_t> plan = chunk_plan(n, m);
  const int64_t n_chunks = (int64_t)plan.size();
  const int slots = (int)std::min<int64_t>(pyro_mech::kSlots, n_chunks);
  for (int s = 0; s < slots; ++s)
    for (size_t i = 0; i < args.size(); ++i)
      if (args[i].host)
        if (int rc = ensure_stage(h, s, i, (size_t)args[i].rows * m * args[i].elem)) return rc;
  auto drain = [&](int code, const std::string& msg) {
    for (int s = 0; s < slots; ++s) cudaStreamSynchronize(h->pipe_stream[s]);
    return fail(code, msg);
  };
  // the pipeline starts after the work already queued on the caller's stream
  if (cudaEventRecord(h->pipe_start, (cudaStream_t)stream) != cudaSuccess) return fail(PYRO_ECUDA, "event record");
  for (int s = 0; s < slots; ++s)
    if (cudaStreamWaitEvent(h->pipe_stream[s], h->pipe_start, 0) != cudaSuccess) return drain(PYRO_ECUDA, "stream wait");
  int64_t p0 = 0;
  for (int64_t c = 0; c < n_chunks; p0 += plan[c], ++c) {
    const int s = (int)(c % slots);
    cudaStream_t st = h->pipe_stream[s];
    const int64_t nc = plan[c];
    for (size_t i = 0; i < args.size(); ++i) {
      if (!args[i].host) continue;
      dev[i] = h->stage[s][i];
      if (!args[i].in) continue;
      const size_t w = (size_t)nc * args[i].elem;
      const char* src = (const char*)args[i].host + (size_t)p0 * args[i].elem;
      cudaError_t e = copy_rows(dev[i], w, src, (size_t)n * args[i].elem, w, args[i].rows, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return drain(PYRO_ECUDA, std::string("H2D copy: ") + cudaGetErrorString(e));
    }
    if (!concurrent && c > 0 && cudaStreamWaitEvent(st, h->pipe_kdone[(c - 1) % slots], 0) != cudaSuccess)
      return drain(PYRO_ECUDA, "stream wait");
    if (int rc = launch(dev, nc, (void*)st)) { for (int q = 0; q < slots; ++q) cudaStreamSynchronize(h->pipe_stream[q]); return rc; }
    if (!concurrent && cudaEventRecord(h->pipe_kdone[s], st) != cudaSuccess) return drain(PYRO_ECUDA, "event record");
    for (size_t i = 0; i < args.size(); ++i) {
      if (!args[i].host || !args[i].out) continue;
      const size_t w = (size_t)nc * args[i].elem;
      char* dst = (char*)const_cast<void*>(args[i].host) + (size_t)p0 * args[i].elem;
      cudaError_t e = copy_rows(dst, (size_t)n * args[i].elem, dev[i], w, w, args[i].rows, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return drain(PYRO_ECUDA, std::string("D2H copy: ") + cudaGetErrorString(e));
    }
  }
  for (int s = 0; s < slots; ++s) {
    cudaError_t e = cudaStreamSynchronize(h->pipe_stream[s]);
    if (e != cudaSuccess) return drain(PYRO_ECUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
  }
  return PYRO_OK;
}

int check_device(const pyro_mech* h) {
  if (!h->module) return fail(PYRO_EINVAL, "mechanism handle was loaded with device=0 (compile only)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(PYRO_ECUDA, "cudaGetDevice failed");
  if (dev != h->device) return fail(PYRO_EINVAL, "mechanism was loaded on device " + std::to_string(h->device) +
                                                   " but the current device is " + std::to_string(dev));
  return PYRO_OK;
}

int launch(const pyro_mech* h, CUfunction f, int64_t n, int blocks_per_sm, unsigned smem, void* stream,
           void** params) {
  int64_t need = (n + h->opt.block - 1) / h->opt.block;
  int64_t cap = (int64_t)h->num_sms * blocks_per_sm;
  unsigned grid = (unsigned)(need < cap ? need : cap);
  if (grid == 0) return PYRO_OK;
  CUresult r = driver().LaunchKernel(f, grid, 1, 1, h->opt.block, 1, 1, smem, as_stream(stream), params, nullptr);
  if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
  return PYRO_OK;
}

int maybe_checked(const pyro_mech* h, void* stream) {
  if (!h->opt.checked) return PYRO_OK;
  int64_t c = 0;
  int rc = pyro_nonconverged(const_cast<pyro_mech*>(h), stream, &c);
  if (rc) return rc;
  if (c) return fail(PYRO_ENOCONV, std::to_string(c) + " point(s) did not converge in the Newton solve");
  return PYRO_OK;
}


// grow the per-block species-array store to `bytes` (allocation at load / first use)
int ensure_store(pyro_mech* h, size_t bytes) {
  if (bytes <= h->store_bytes) return PYRO_OK;
  if (h->d_store) cudaFree(h->d_store);
  h->d_store = nullptr;
  h->store_bytes = 0;
  cudaError_t e = cudaMalloc(&h->d_store, bytes);
  if (e != cudaSuccess) return fail(PYRO_ECUDA, std::string("species-array store allocation: ") + cudaGetErrorString(e));
  h->store_bytes = bytes;
  return PYRO_OK;
}

const char* group_kernel(const std::string& g) {
  return g == "jvp" ? "pyro_jvp" : g == "vjp" ? "pyro_vjp" : g == "jad" ? "pyro_jacobian_adiabatic"
       : g == "cn" ? "pyro_cn_assemble" : g == "tr" ? "pyro_transport" : g == "wfwd" ? "pyro_omega_warp"
       : g == "wjvp" ? "pyro_jvp_warp" : g == "wvjp" ? "pyro_vjp_warp" : g == "wjac" ? "pyro_jacobian_cta"
       : g == "wjad" ? "pyro_jacobian_adiabatic_cta" : "pyro_jacobian";
}

// Compile (in parallel threads, cached on disk) and load the named derivative
// kernel groups that are not loaded yet.
int ensure_groups(pyro_mech* h, const std::vector<std::string>& names) {
  std::lock_guard<std::mutex> lock(h->group_mu);
  std::vector<std::string> todo;
  for (auto& g : names) {
    auto& G = h->groups[g];
    if (G.failed) return fail(PYRO_ECOMPILE, G.err);
    if (!G.module && !(h->module == nullptr && G.blocks_per_sm < 0)) todo.push_back(g);
  }
  if (todo.empty()) return PYRO_OK;
  std::vector<std::vector<char>> cubins(todo.size());
  std::vector<int> rcs(todo.size(), PYRO_OK);
  std::vector<std::string> errs(todo.size());
  std::vector<std::thread> th;
  for (size_t i = 0; i < todo.size(); ++i) {
    th.emplace_back([&, i] {
      rcs[i] = compile_cached(h->emitted.group_sources.at(todo[i]), h->opt.cache, cubins[i]);
      if (rcs[i]) errs[i] = pyro_last_error();
    });
  }
  for (auto& t : th) t.join();
  if (!h->module) {   // compile-only handle: record the build, load nothing
    for (size_t i = 0; i < todo.size(); ++i) {
      auto& G = h->groups[todo[i]];
      if (rcs[i]) { G.failed = true; G.err = errs[i]; return fail(rcs[i], errs[i]); }
      G.blocks_per_sm = -1;
      h->emitted.stats[todo[i] + "_cubin_bytes"] = (double)cubins[i].size();
    }
    return PYRO_OK;
  }
  Driver& d = driver();
  for (size_t i = 0; i < todo.size(); ++i) {
    auto& G = h->groups[todo[i]];
    if (rcs[i]) { G.failed = true; G.err = errs[i]; return fail(rcs[i], errs[i]); }
    CUresult r = d.ModuleLoadData(&G.module, cubins[i].data());
    if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "cuModuleLoadData: " + cu_err(r));
    r = d.ModuleGetFunction(&G.f, G.module, group_kernel(todo[i]));
    if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, std::string("missing kernel ") + group_kernel(todo[i]));
    if (todo[i] == "tr") { G.block = pyro::kTransportBlock; G.smem = h->emitted.smem_dyn_bytes_transport; }
    if (todo[i][0] == 'w') {
      G.block = 32 * h->emitted.warp_wpb.at(todo[i]);
      G.smem = h->emitted.smem_dyn_bytes_warp.at(todo[i]);
    }
    if (todo[i] == "jac" || todo[i] == "jad" || todo[i] == "cn") G.smem = h->emitted.smem_dyn_bytes_jac;
    const int smem = G.smem >= 0 ? G.smem : h->emitted.smem_dyn_bytes_deriv;
    const int blk = G.block > 0 ? G.block : h->opt.deriv_block;
    r = d.FuncSetAttribute(G.f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, smem);
    if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "shared memory request: " + cu_err(r));
    int nb = 0;
    r = d.Occupancy(&nb, G.f, blk, smem);
    if (r != CUDA_SUCCESS || nb < 1) return fail(PYRO_ECUDA, std::string(group_kernel(todo[i])) + " does not fit on an SM");
    G.blocks_per_sm = nb;
    h->emitted.stats[todo[i] + "_blocks_per_sm"] = nb;
    if (todo[i] == "wjac" || todo[i] == "wjad") {
      // persistent grid of the clusters that fit at once (a cluster's blocks share a GPC)
      CUlaunchConfig cfg;
      std::memset(&cfg, 0, sizeof(cfg));
      cfg.gridDimX = (unsigned)(pyro::kJacCluster * h->num_sms);
      cfg.gridDimY = cfg.gridDimZ = 1;
      cfg.blockDimX = (unsigned)blk;
      cfg.blockDimY = cfg.blockDimZ = 1;
      cfg.sharedMemBytes = (unsigned)smem;
      int ncl = 0;
      r = d.MaxActiveClusters(&ncl, G.f, &cfg);
      if (r != CUDA_SUCCESS || ncl < 1) return fail(PYRO_ECUDA, std::string(group_kernel(todo[i])) + ": no cluster fits");
      G.clusters = ncl;
      h->emitted.stats[todo[i] + "_active_clusters"] = ncl;
    }
    if (h->emitted.stats["deriv_store_global"] > 0 && todo[i] != "jac" && todo[i] != "jad" && todo[i] != "cn" &&
        todo[i][0] != 'w') {
      size_t bytes = (size_t)h->num_sms * nb * 4 * h->m.n_species() * h->opt.deriv_block * sizeof(double);
      cudaError_t e = cudaMalloc(&G.store, bytes);
      if (e != cudaSuccess) return fail(PYRO_ECUDA, std::string("species-array store allocation: ") + cudaGetErrorString(e));
    }
    if (todo[i] == "cn") {
      for (const char* nm : {"pyro_cn_prep", "pyro_cn_solve", "pyro_cn_finish", "pyro_cn_residual"}) {
        if (h->emitted.stats["cn_residual_kernel"] <= 0 && std::string(nm) == "pyro_cn_residual") continue;
        CUfunction f = nullptr;
        r = d.ModuleGetFunction(&f, G.module, nm);
        if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, std::string("missing kernel ") + nm);
        G.fn[nm] = f;
      }
      const int ssm = h->emitted.smem_dyn_bytes_cn_solve;
      r = d.FuncSetAttribute(G.fn["pyro_cn_solve"], CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, ssm);
      if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "shared memory request (Crank-Nicolson solve): " + cu_err(r));
      int sb = 0;
      r = d.Occupancy(&sb, G.fn["pyro_cn_solve"], 32 * h->emitted.cn_solve_warps, ssm);
      if (r != CUDA_SUCCESS || sb < 1) return fail(PYRO_ECUDA, "pyro_cn_solve does not fit on an SM");
      G.solve_blocks_per_sm = sb;
      h->emitted.stats["cn_solve_blocks_per_sm"] = sb;
      if (h->emitted.stats["cn_residual_kernel"] > 0) {   // chord iterations
        const int rsm = 2 * h->m.n_species() * h->opt.deriv_block * (int)sizeof(double);
        r = d.FuncSetAttribute(G.fn["pyro_cn_residual"], CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, rsm);
        if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "shared memory request (Crank-Nicolson residual): " + cu_err(r));
        int rb = 0;
        r = d.Occupancy(&rb, G.fn["pyro_cn_residual"], h->opt.deriv_block, rsm);
        if (r != CUDA_SUCCESS || rb < 1) return fail(PYRO_ECUDA, "pyro_cn_residual does not fit on an SM");
        G.residual_blocks_per_sm = rb;
      }
    }
    h->emitted.stats[todo[i] + "_cubin_bytes"] = (double)cubins[i].size();
  }
  return PYRO_OK;
}

// grow the per-block scratch of the Jacobian-type kernels (per-reaction partials)
int ensure_jac_scratch(pyro_mech* h, const pyro_mech::Group& G, int64_t n) {
  std::lock_guard<std::mutex> lock(h->mu);
  int64_t need = (n + h->opt.deriv_block - 1) / h->opt.deriv_block;
  int64_t grid = std::min<int64_t>(need, (int64_t)h->num_sms * G.blocks_per_sm);
  size_t bytes = (size_t)grid * h->emitted.jac_slots * h->opt.deriv_block * sizeof(double);
  if (bytes > h->jac_scratch_bytes) {
    if (h->d_jac_scratch) cudaFree(h->d_jac_scratch);
    h->d_jac_scratch = nullptr;
    h->jac_scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&h->d_jac_scratch, bytes);
    if (e != cudaSuccess) return fail(PYRO_ECUDA, std::string("Jacobian scratch allocation: ") + cudaGetErrorString(e));
    h->jac_scratch_bytes = bytes;
  }
  return PYRO_OK;
}

// warp-per-state kernels: one state per warp, a persistent grid of the resident blocks
int launch_warp(const pyro_mech* h, const pyro_mech::Group& G, int64_t n, void* stream, void** params) {
  const int wpb = G.block / 32;
  int64_t need = (n + wpb - 1) / wpb;
  int64_t cap = (int64_t)h->num_sms * G.blocks_per_sm;
  unsigned grid = (unsigned)(need < cap ? need : cap);
  if (grid == 0) return PYRO_OK;
  CUresult r = driver().LaunchKernel(G.f, grid, 1, 1, G.block, 1, 1, G.smem, as_stream(stream), params, nullptr);
  if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
  return PYRO_OK;
}

// block-per-state kernels (dense Jacobians of variant=warp): one state per block
// and iteration, a persistent grid of the resident blocks
int launch_cta(const pyro_mech* h, const pyro_mech::Group& G, int64_t n, void* stream, void** params) {
  // clusters of kJacCluster blocks: the grid is a multiple of the cluster size
  const int64_t CLs = pyro::kJacCluster;
  const int64_t cap = CLs * G.clusters;
  const int64_t need = (n + CLs - 1) / CLs * CLs;
  unsigned grid = (unsigned)(need < cap ? need : cap);
  if (grid == 0) return PYRO_OK;
  CUresult r = driver().LaunchKernel(G.f, grid, 1, 1, G.block, 1, 1, G.smem, as_stream(stream), params, nullptr);
  if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
  return PYRO_OK;
}

// the dense Jacobian groups of a handle: block per state (variant=warp, where
// emitted) or thread per state
std::string jac_group(const pyro_mech* h, bool adiabatic) {
  pyro_mech* m = const_cast<pyro_mech*>(h);
  if (h->opt.warp && m->emitted.stats[adiabatic ? "jacobian_adiabatic_cta" : "jacobian_cta"] > 0)
    return adiabatic ? "wjad" : "wjac";
  return adiabatic ? "jad" : "jac";
}

int launch_deriv(const pyro_mech* h, const pyro_mech::Group& G, int64_t n, void* stream, void** params) {
  const int blk = G.block > 0 ? G.block : h->opt.deriv_block;
  const int smem = G.smem >= 0 ? G.smem : h->emitted.smem_dyn_bytes_deriv;
  int64_t need = (n + blk - 1) / blk;
  int64_t cap = (int64_t)h->num_sms * G.blocks_per_sm;
  unsigned grid = (unsigned)(need < cap ? need : cap);
  if (grid == 0) return PYRO_OK;
  CUresult r = driver().LaunchKernel(G.f, grid, 1, 1, blk, 1, 1, smem, as_stream(stream), params, nullptr);
  if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
  return PYRO_OK;
}
}  // namespace

extern "C" {

const char* pyro_last_error(void) { return g_last_error.c_str(); }

int pyro_version(void) { return 100; }

int pyro_mech_load(const char* mech_path, const char* options, pyro_mech** out) {
  if (!mech_path || !out) return fail(PYRO_EINVAL, "null argument");
  *out = nullptr;
  auto* h = new pyro_mech();
  std::string err;
  if (!parse_options(options, h->opt, err)) { delete h; return fail(PYRO_EINVAL, err); }
  if (!parse_mechanism_file(mech_path, h->m, err)) { delete h; return fail(PYRO_EMECH, err); }
  if (!validate_mechanism(h->m, err)) { delete h; return fail(PYRO_EMECH, err); }
  if (h->opt.warp && !pyro::warp_supported(h->m, &err)) {
    delete h;
    return fail(PYRO_EINVAL, err);
  }
  for (auto& s : h->m.species) h->W.push_back(s.W);
  EmitOptions eo;
  eo.block = h->opt.block;
  eo.min_blocks = h->opt.block <= 64 ? 4 : (h->opt.block <= 128 ? 2 : 1);
  eo.mixed_newton = h->opt.mixed;
  eo.deriv_block = h->opt.deriv_block;
  eo.exp_ops = h->opt.exp_ops;
  eo.warp_exp_ops = h->opt.warp_exp_ops;
  eo.exp_call = h->opt.exp_call;
  {
    const int N = h->m.n_species();
    const size_t lim = 160 * 1024;
    eo.gstore = h->opt.store == 2 || (h->opt.store == 0 && (size_t)2 * N * eo.block * 8 > lim);
    eo.dgstore = h->opt.store == 2 || (h->opt.store == 0 && (size_t)4 * N * eo.deriv_block * 8 > lim);
    eo.acc_mem = N > 64;
    eo.jac_table = h->opt.jac_rows == 2 || (h->opt.jac_rows == 0 && N > 64);
    eo.cn_residual = h->opt.cn_chord || !eo.jac_table;   // large mechanisms: only where chord asks for it
    if (eo.gstore && eo.block > 64) eo.min_blocks = 1;
  }
  h->emitted = emit_module(h->m, eo);

  // compile (or fetch from the cache)
  std::vector<char> cubin;
  if (int rc = compile_cached(h->emitted.source, h->opt.cache, cubin)) { delete h; return rc; }
  h->emitted.stats["cubin_bytes"] = (double)cubin.size();
  if (!h->opt.device) { *out = h; return PYRO_OK; }
  Driver& d = driver();
  if (!d.ok) { delete h; return fail(PYRO_ECUDA, d.err); }
  cudaError_t ce = cudaFree(0);   // make sure a context is current
  if (ce != cudaSuccess) { delete h; return fail(PYRO_ECUDA, std::string("CUDA init: ") + cudaGetErrorString(ce)); }
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device);
  if (major * 10 + minor != 103) {
    delete h;
    return fail(PYRO_ECUDA, "libpyro is built for sm_103a (GB300); device has sm_" + std::to_string(major * 10 + minor));
  }

  CUresult r = d.ModuleLoadData(&h->module, cubin.data());
  if (r != CUDA_SUCCESS) { delete h; return fail(PYRO_ECUDA, "cuModuleLoadData: " + cu_err(r)); }
  struct { const char* name; CUfunction* f; } fns[] = {
      {"pyro_omega", &h->f_omega}, {"pyro_temperature", &h->f_temperature}, {"pyro_energy", &h->f_energy},
      {"pyro_density", &h->f_density}, {"pyro_math", &h->f_math}, {"pyro_enthalpy", &h->f_enthalpy},
      {"pyro_temperature_h", &h->f_temperature_h}};
  for (auto& q : fns) {
    r = d.ModuleGetFunction(q.f, h->module, q.name);
    if (r != CUDA_SUCCESS) { pyro_mech_free(h); return fail(PYRO_ECUDA, std::string("missing kernel ") + q.name); }
  }
  if (h->emitted.stats["mlp_supported"] > 0) {
    if (d.ModuleGetFunction(&h->f_mlp_guess, h->module, "pyro_mlp_guess") != CUDA_SUCCESS ||
        d.ModuleGetFunction(&h->f_temperature_mlp, h->module, "pyro_temperature_mlp") != CUDA_SUCCESS) {
      pyro_mech_free(h);
      return fail(PYRO_ECUDA, "missing learned-guess kernels");
    }
  }
  int smem = h->emitted.smem_dyn_bytes_omega;
  r = d.FuncSetAttribute(h->f_omega, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, smem);
  if (r != CUDA_SUCCESS) { pyro_mech_free(h); return fail(PYRO_ECUDA, "shared memory request of " + std::to_string(smem) + " B: " + cu_err(r)); }
  int nb = 0;
  r = d.Occupancy(&nb, h->f_omega, h->opt.block, smem);
  if (r != CUDA_SUCCESS || nb < 1) { pyro_mech_free(h); return fail(PYRO_ECUDA, "omega kernel does not fit on an SM"); }
  h->omega_blocks_per_sm = nb;
  h->emitted.stats["omega_blocks_per_sm"] = nb;
  if (h->emitted.stats["omega_store_global"] > 0) {
    size_t bytes = (size_t)h->num_sms * nb * 2 * h->m.n_species() * h->opt.block * sizeof(double);
    if (int rc = ensure_store(h, bytes)) { pyro_mech_free(h); return rc; }
  }
  if (h->opt.warp) {
    // the emitted warp-per-state forward kernel (compiled now, cached on disk)
    if (int rc = ensure_groups(h, {"wfwd"})) { pyro_mech_free(h); return rc; }
    h->emitted.stats["variant_warp"] = 1;
  }
  if (cudaMalloc(&h->d_fail, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(h->d_fail, 0, sizeof(unsigned long long)) != cudaSuccess) {
    pyro_mech_free(h);
    return fail(PYRO_ECUDA, "failure counter allocation");
  }
  // the no-allocation entry point's static scratch: its module is loaded (and its
  // device memory taken) here, where allocating is allowed, not in its first call
  if (int rc = pyro::noalloc_prepare_device()) { pyro_mech_free(h); return rc; }
  *out = h;
  return PYRO_OK;
}

void pyro_mech_free(pyro_mech* h) {
  if (!h) return;
  if (h->module && driver().ModuleUnload) driver().ModuleUnload(h->module);
  if (h->d_fail) cudaFree(h->d_fail);
  if (h->d_jac_scratch) cudaFree(h->d_jac_scratch);
  if (h->d_cn) cudaFree(h->d_cn);
  if (h->d_store) cudaFree(h->d_store);
  if (h->mlp) pyro::mlp_free(h->mlp);
  if (h->mlp_norm_dev) cudaFree(h->mlp_norm_dev);
  for (auto& g : h->groups) {
    if (g.second.module && driver().ModuleUnload) driver().ModuleUnload(g.second.module);
    if (g.second.store) cudaFree(g.second.store);
  }
  for (int s = 0; s < pyro_mech::kSlots; ++s) {
    for (void* p : h->stage[s]) if (p) cudaFree(p);
    if (h->pipe_stream[s]) cudaStreamDestroy(h->pipe_stream[s]);
    if (h->pipe_kdone[s]) cudaEventDestroy(h->pipe_kdone[s]);
  }
  if (h->pipe_start) cudaEventDestroy(h->pipe_start);
  delete h;
}

int pyro_mech_info(const pyro_mech* h, int* ns, int* nr, const double** W) {
  if (!h) return fail(PYRO_EINVAL, "null mechanism");
  if (ns) *ns = h->m.n_species();
  if (nr) *nr = h->m.n_reactions();
  if (W) *W = h->W.data();
  return PYRO_OK;
}

int pyro_mech_stat(const pyro_mech* h, const char* key, double* value) {
  if (!h || !key || !value) return fail(PYRO_EINVAL, "null argument");
  auto it = h->emitted.stats.find(key);
  if (it == h->emitted.stats.end()) return fail(PYRO_EINVAL, std::string("unknown stat '") + key + "'");
  *value = it->second;
  return PYRO_OK;
}

const char* pyro_mech_source(const pyro_mech* h) { return h ? h->emitted.source.c_str() : ""; }

int pyro_density(const pyro_mech* hc, int64_t n, const double* p, const double* T, const double* Y,
                 double* rho, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!p || !T || !Y || !rho))) return fail(PYRO_EINVAL, "pyro_density: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{p, 1, 8, true, false}, {T, 1, 8, true, false}, {Y, NS, 8, true, false}, {rho, 1, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3]};
                     return launch(h, h->f_density, nc, 8, 0, st, params);
                   }, true);
}

int pyro_internal_energy(const pyro_mech* hc, int64_t n, const double* T, const double* Y, double* e,
                         double* cv, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!T || !Y || !e))) return fail(PYRO_EINVAL, "pyro_internal_energy: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{T, 1, 8, true, false}, {Y, NS, 8, true, false}, {e, 1, 8, false, true}, {cv, 1, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3]};
                     return launch(h, h->f_energy, nc, 8, 0, st, params);
                   }, true);
}

int pyro_enthalpy(const pyro_mech* hc, int64_t n, const double* T, const double* Y, double* hm, double* cp,
                  void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!T || !Y || !hm))) return fail(PYRO_EINVAL, "pyro_enthalpy: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{T, 1, 8, true, false}, {Y, NS, 8, true, false}, {hm, 1, 8, false, true}, {cp, 1, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3]};
                     return launch(h, h->f_enthalpy, nc, 8, 0, st, params);
                   }, true);
}

int pyro_temperature_enthalpy(const pyro_mech* hc, int64_t n, const double* hm, const double* Y,
                              const double* T_guess, double* T_out, int32_t* iters, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!hm || !Y || !T_out)))
    return fail(PYRO_EINVAL, "pyro_temperature_enthalpy: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const int64_t NS = h->m.n_species();
  int rc = with_args(h, n, {{hm, 1, 8, true, false}, {Y, NS, 8, true, false}, {T_guess, 1, 8, true, false},
                            {T_out, 1, 8, false, true}, {iters, 1, 4, false, true}},
                     stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                       long long nn = nc;
                       double Tg = 1200.0, tol = 1e-10;
                       int max_iter = 50;
                       void* params[] = {&nn, &d[0], &d[1], &d[2], &Tg, &max_iter, &tol, &d[3], &d[4], &h->d_fail};
                       return launch(h, h->f_temperature_h, nc, 8, 0, st, params);
                     }, true);
  if (rc) return rc;
  return maybe_checked(h, stream);
}

int pyro_temperature(const pyro_mech* hc, int64_t n, const double* e, const double* Y, const double* T_guess,
                     int guess_mode, double* T_out, int32_t* iters, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!e || !Y || !T_out))) return fail(PYRO_EINVAL, "pyro_temperature: bad arguments");
  if (guess_mode != 0 && guess_mode != 1) return fail(PYRO_EINVAL, "guess_mode must be 0 or 1");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  if (guess_mode == 1 && !pyro::mlp_ready(h->mlp)) return fail(PYRO_ENOMLP, "no learned initial guess is loaded");
  const int64_t NS = h->m.n_species();
  int rc = with_args(h, n, {{e, 1, 8, true, false}, {Y, NS, 8, true, false}, {T_guess, 1, 8, true, false},
                         {T_out, 1, 8, false, true}, {iters, 1, 4, false, true}},
                     stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                       long long nn = nc;
                       double Tg = 1200.0, tol = 1e-10;
                       int max_iter = 50;
                       if (guess_mode == 1) {
                         const void* wb = pyro::mlp_device_bf16(h->mlp);
                         const float* wf = pyro::mlp_device_params(h->mlp);
                         const float* nm = h->mlp_norm_dev;
                         void* pm[] = {&nn, &d[0], &d[1], &wb, &wf, &nm, &max_iter, &tol, &d[3], &d[4], &h->d_fail};
                         return launch(h, h->f_temperature_mlp, nc, 8, 0, st, pm);
                       }
                       void* params[] = {&nn, &d[0], &d[1], &d[2], &Tg, &max_iter, &tol, &d[3], &d[4], &h->d_fail};
                       return launch(h, h->f_temperature, nc, 8, 0, st, params);
                     }, true);
  if (rc) return rc;
  return maybe_checked(h, stream);
}

int pyro_net_production_rates(const pyro_mech* hc, int64_t n, const double* rho, const double* T_or_e,
                              int input_is_energy, const double* Y, double* T_out, double* omega,
                              void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!rho || !T_or_e || !Y || !omega)))
    return fail(PYRO_EINVAL, "pyro_net_production_rates: bad arguments");
  if (input_is_energy && !T_out) return fail(PYRO_EINVAL, "T_out is required when input_is_energy != 0");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const int64_t NS = h->m.n_species();
  int rc = with_args(h, n, {{rho, 1, 8, true, false}, {T_or_e, 1, 8, true, false}, {Y, NS, 8, true, false},
                         {input_is_energy ? T_out : nullptr, 1, 8, false, true}, {omega, NS, 8, false, true}},
                     stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                       long long nn = nc;
                       int em = input_is_energy ? 1 : 0;
                       double Tg = 1200.0, tol = 1e-10;
                       int max_iter = 50;
                       void* params[] = {&nn, &d[0], &d[1], &em, &d[2], &d[3], &d[4], &Tg, &max_iter, &tol, &h->d_fail,
                                         &h->d_store};
                       if (h->opt.warp) return launch_warp(h, h->groups["wfwd"], nc, st, params);
                       return launch(h, h->f_omega, nc, h->omega_blocks_per_sm, h->emitted.smem_dyn_bytes_omega,
                                     st, params);
                     }, h->opt.warp || h->emitted.stats["omega_store_global"] <= 0);   // no per-block global scratch
  if (rc) return rc;
  return input_is_energy ? maybe_checked(h, stream) : PYRO_OK;
}


int pyro_mech_prepare(const pyro_mech* hc, const char* kernels) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h) return fail(PYRO_EINVAL, "null mechanism");
  std::string k = kernels ? kernels : "all";
  std::vector<std::string> names;
  if (k == "all") {
    names = {h->opt.warp ? "wjvp" : "jvp", h->opt.warp ? "wvjp" : "vjp", jac_group(h, false)};
  }
  else {
    std::string item;
    std::stringstream ss(k);
    while (std::getline(ss, item, ',')) {
      if (item == "jvp" || item == "vjp") names.push_back(h->opt.warp ? "w" + item : item);
      else if (item == "jacobian" || item == "jac") names.push_back(jac_group(h, false));
      else if (item == "jacobian_adiabatic" || item == "jad") names.push_back(jac_group(h, true));
      else if (item == "cn" || item == "crank_nicolson") names.push_back("cn");
      else if (item == "warp" || item == "wfwd") names.push_back("wfwd");
      else if (item == "transport" || item == "tr") {
        if (h->emitted.stats["has_transport"] <= 0) return fail(PYRO_EMECH, "the mechanism has no transport section");
        names.push_back("tr");
      }
      else if (!item.empty()) return fail(PYRO_EINVAL, "unknown kernel group '" + item + "'");
    }
  }
  return ensure_groups(h, names);
}

int pyro_jvp(const pyro_mech* hc, int64_t n, const double* rho, const double* T, const double* Y,
             const double* d_rho, const double* d_T, const double* d_Y, double* d_omega, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!rho || !T || !Y || !d_rho || !d_T || !d_Y || !d_omega)))
    return fail(PYRO_EINVAL, "pyro_jvp: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const std::string g = h->opt.warp ? "wjvp" : "jvp";   // one warp or one thread per state
  if (int rc = ensure_groups(h, {g})) return rc;
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{rho, 1, 8, true, false}, {T, 1, 8, true, false}, {Y, NS, 8, true, false}, {d_rho, 1, 8, true, false},
                       {d_T, 1, 8, true, false}, {d_Y, NS, 8, true, false}, {d_omega, NS, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3], &d[4], &d[5], &d[6], &h->groups[g].store};
                     if (h->opt.warp) return launch_warp(h, h->groups[g], nc, st, params);
                     return launch_deriv(h, h->groups[g], nc, st, params);
                   }, h->opt.warp);
}

int pyro_vjp(const pyro_mech* hc, int64_t n, const double* rho, const double* T, const double* Y,
             const double* omega_bar, double* rho_bar, double* T_bar, double* Y_bar, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!rho || !T || !Y || !omega_bar || !rho_bar || !T_bar || !Y_bar)))
    return fail(PYRO_EINVAL, "pyro_vjp: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const std::string g = h->opt.warp ? "wvjp" : "vjp";
  if (int rc = ensure_groups(h, {g})) return rc;
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{rho, 1, 8, true, false}, {T, 1, 8, true, false}, {Y, NS, 8, true, false}, {omega_bar, NS, 8, true, false},
                       {rho_bar, 1, 8, false, true}, {T_bar, 1, 8, false, true}, {Y_bar, NS, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3], &d[4], &d[5], &d[6], &h->groups[g].store};
                     if (h->opt.warp) return launch_warp(h, h->groups[g], nc, st, params);
                     return launch_deriv(h, h->groups[g], nc, st, params);
                   }, h->opt.warp);
}

int pyro_jacobian(const pyro_mech* hc, int64_t n, const double* rho, const double* T, const double* Y,
                  double* J, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!rho || !T || !Y || !J))) return fail(PYRO_EINVAL, "pyro_jacobian: bad arguments");
  if (h && h->emitted.stats["jacobian_supported"] <= 0)
    return fail(PYRO_EINVAL, "the dense Jacobian kernels need all species to share one NASA-7 T_mid");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const std::string g = jac_group(h, false);
  if (int rc = ensure_groups(h, {g})) return rc;
  const pyro_mech::Group& G = h->groups[g];
  const bool cta = g[0] == 'w';
  int NP = h->m.n_species() + 1;
  const int64_t NS = h->m.n_species();
  if (!cta)
    if (int rc = ensure_jac_scratch(h, G, n)) return rc;
  return with_args(h, n, {{rho, 1, 8, true, false}, {T, 1, 8, true, false}, {Y, NS, 8, true, false}, {J, (int64_t)NP * NP, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3], &h->d_jac_scratch};
                     return cta ? launch_cta(h, G, nc, st, params) : launch_deriv(h, G, nc, st, params);
                   }, cta);
}


int pyro_transport(const pyro_mech* hc, int64_t n, const double* T, const double* Y, double* mu, double* kappa,
                   double* D_mix, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!T || !Y || (!mu && !kappa && !D_mix))))
    return fail(PYRO_EINVAL, "pyro_transport: bad arguments");
  if (h->emitted.stats["has_transport"] <= 0) return fail(PYRO_EMECH, "the mechanism has no transport section");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  if (int rc = ensure_groups(h, {"tr"})) return rc;
  pyro_mech::Group& G = h->groups["tr"];
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{T, 1, 8, true, false}, {Y, NS, 8, true, false}, {mu, 1, 8, false, true},
                          {kappa, 1, 8, false, true}, {D_mix, NS, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3], &d[4], &G.store};
                     return launch_deriv(h, G, nc, st, params);
                   });
}

int pyro_jacobian_adiabatic(const pyro_mech* hc, int64_t n, const double* rho, const double* T, const double* Y,
                            double* J, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!rho || !T || !Y || !J)))
    return fail(PYRO_EINVAL, "pyro_jacobian_adiabatic: bad arguments");
  if (h && h->emitted.stats["jacobian_supported"] <= 0)
    return fail(PYRO_EINVAL, "the dense Jacobian kernels need all species to share one NASA-7 T_mid");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  const std::string g = jac_group(h, true);
  if (int rc = ensure_groups(h, {g})) return rc;
  const pyro_mech::Group& G = h->groups[g];
  const bool cta = g[0] == 'w';
  const int64_t NS = h->m.n_species();
  if (!cta)
    if (int rc = ensure_jac_scratch(h, G, n)) return rc;
  return with_args(h, n, {{rho, 1, 8, true, false}, {T, 1, 8, true, false}, {Y, NS, 8, true, false}, {J, NS * NS, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     void* params[] = {&nn, &d[0], &d[1], &d[2], &d[3], &h->d_jac_scratch};
                     return cta ? launch_cta(h, G, nc, st, params) : launch_deriv(h, G, nc, st, params);
                   }, cta);
}

namespace {
// States per chunk of the Crank-Nicolson work arrays (Newton matrix N^2 doubles
// per state): at most 8 GiB, a multiple of the matrix group size.  Chunks run one
// after another and each ends in a tail of slowly converging states that keeps
// only a few warps busy, so fewer, larger chunks are faster.
// FP32 words per state of the kept factorisation (chord iterations): LU rows of
// the solve kernel's leading dimension, pivots, row exponents.
int64_t cn_fac_words(const pyro_mech* h) {
  const int64_t N = h->m.n_species();
  const int64_t half = (N + 1) / 2, lda = half % 2 == 1 ? 2 * half : 2 * half + 2;
  return N * lda + 2 * N;
}

size_t cn_bytes_per_state(const pyro_mech* h) {
  const int64_t N = h->m.n_species();
  return (size_t)(N * N + 2 * N + 3) * sizeof(double) + (h->opt.cn_chord ? (size_t)cn_fac_words(h) * 4 : 0);
}

int64_t cn_chunk(const pyro_mech* h, int64_t n) {
  const int64_t Gs = pyro::kCnGroup;
  const size_t per_state = cn_bytes_per_state(h);
  int64_t m = std::max<int64_t>(4096, (int64_t)(((size_t)8 << 30) / per_state));
  m = std::min<int64_t>(m, (n + Gs - 1) / Gs * Gs);
  return (m + Gs - 1) / Gs * Gs;
}

// Allocate (grow) the Crank-Nicolson work arrays and the Jacobian scratch for
// calls of up to n states.
int cn_reserve(pyro_mech* h, int64_t n) {
  const int64_t N = h->m.n_species();
  const int64_t m = cn_chunk(h, n);
  if (int rc = ensure_jac_scratch(h, h->groups["cn"], m)) return rc;
  std::lock_guard<std::mutex> lock(h->mu);
  const size_t bytes = (size_t)m * cn_bytes_per_state(h) + 64;   // + counters and alignment
  (void)N;
  if (bytes > h->cn_bytes) {
    if (h->d_cn) cudaFree(h->d_cn);
    h->d_cn = nullptr;
    h->cn_bytes = 0;
    cudaError_t e = cudaMalloc(&h->d_cn, bytes);
    if (e != cudaSuccess) return fail(PYRO_ECUDA, std::string("Crank-Nicolson scratch allocation: ") + cudaGetErrorString(e));
    h->cn_bytes = bytes;
  }
  return PYRO_OK;
}

// Crank-Nicolson step over `cnt` states of arrays with row stride `ld` (pointers
// already offset to the first state), in chunks of cn_chunk states; the work
// arrays must have been reserved (cn_reserve) for at least cnt states.
int cn_run(pyro_mech* h, int64_t cnt, int64_t ld, double dt, const double* rho, const double* Tin,
           const double* Yin, double tol, int max_newton, int refine, double* Tout, double* Yout, int32_t* iters,
           void* stream) {
  const pyro_mech::Group& G = h->groups["cn"];
  const int64_t N = h->m.n_species();
  const int64_t m = cn_chunk(h, cnt);
  double* dA = (double*)h->d_cn;                 // [m/G][N^2][G]
  double* dc = dA + (size_t)m * N * N;           // [N][m]
  double* db = dc + (size_t)m * N;               // [N][m]
  double* de = db + (size_t)m * N;               // [m]
  int* dstate = (int*)(de + m);                  // [m]
  int* dit = dstate + m;                         // [m]
  int* dlist[2] = {dit + m, dit + 2 * m};        // active-state lists [m], built alternately
  int* dcount[2] = {dit + 3 * m, dit + 3 * m + 1};
  float* dfac = h->opt.cn_chord ? (float*)(dcount[1] + 1) : nullptr;   // [m][fac words] (chord)
  if (dfac) dfac = (float*)(((uintptr_t)dfac + 15) & ~(uintptr_t)15);
  Driver& d = driver();
  const int bd = h->opt.deriv_block;
  double Tg_tol = 1e-10;
  int t_iter = 50;
  for (int64_t p0 = 0; p0 < cnt; p0 += m) {
    long long nc = std::min<int64_t>(m, cnt - p0), nld = ld;
    const double* rho_c = rho + p0;
    const double* Tin_c = Tin + p0;
    const double* Yin_c = Yin + p0;
    double* Tout_c = Tout + p0;
    double* Yout_c = Yout + p0;
    int32_t* it_c = iters ? iters + p0 : nullptr;
    unsigned gs = (unsigned)std::min<int64_t>((nc + bd - 1) / bd, (int64_t)h->num_sms * 8);
    void* pp[] = {&nc, &nld, &Tin_c, &Yin_c, &Tout_c, &Yout_c, &de, &dstate, &dit, &dlist[0], &dcount[0]};
    CUresult r = d.LaunchKernel(G.fn.at("pyro_cn_prep"), gs, 1, 1, bd, 1, 1, 0, as_stream(stream), pp, nullptr);
    if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
    const int64_t Ws = h->emitted.cn_solve_warps;   // states per block of the solve
    unsigned gsolve = (unsigned)std::min<int64_t>((nc + Ws - 1) / Ws, (int64_t)h->num_sms * G.solve_blocks_per_sm);
    const bool chord = h->opt.cn_chord;
    unsigned gres = (unsigned)std::min<int64_t>((nc + bd - 1) / bd, (int64_t)h->num_sms * G.residual_blocks_per_sm);
    const unsigned rsm = (unsigned)(2 * N * bd * sizeof(double));
    for (int it = 0; it <= max_newton; ++it) {
      int* li = dlist[it & 1];
      int* lo = dlist[(it + 1) & 1];
      int* ci = dcount[it & 1];
      int* co = dcount[(it + 1) & 1];
      int mode = chord ? (it % h->opt.cn_refresh == 0 ? 1 : 2) : 0;
      int a_at_state = chord ? 1 : 0;
      if (mode == 2) {   // chord: right-hand side only, the first iterate's matrix is kept
        void* pr[] = {&nc, &nld, &rho_c, &de, &Yout_c, &dc, &Tout_c, &dstate, &dt, &t_iter, &Tg_tol, &db,
                      &h->d_fail, &li, &ci, &co};
        r = d.LaunchKernel(G.fn.at("pyro_cn_residual"), gres, 1, 1, bd, 1, 1, rsm, as_stream(stream), pr, nullptr);
        if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
      } else {
        void* pa[] = {&nc, &nld, &rho_c, &de, &Yout_c, &dc, &Tout_c, &dstate, &dt, &t_iter, &Tg_tol, &dA, &db,
                      &h->d_jac_scratch, &h->d_fail, &li, &ci, &co, &a_at_state};
        if (int rc = launch_deriv(h, G, nc, stream, pa)) return rc;
      }
      void* ps[] = {&nc, &nld, &dA, &db, &Yout_c, &dstate, &dit, &tol, &max_newton, &refine, &h->d_fail,
                    &li, &ci, &lo, &co, &mode, &dfac};
      r = d.LaunchKernel(G.fn.at("pyro_cn_solve"), gsolve, 1, 1, 32 * (unsigned)Ws, 1, 1,
                         h->emitted.smem_dyn_bytes_cn_solve, as_stream(stream), ps, nullptr);
      if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
    }
    void* pf[] = {&nc, &nld, &de, &Yout_c, &Tout_c, &dstate, &dit, &it_c, &t_iter, &Tg_tol, &h->d_fail};
    r = d.LaunchKernel(G.fn.at("pyro_cn_finish"), gs, 1, 1, bd, 1, 1, 0, as_stream(stream), pf, nullptr);
    if (r != CUDA_SUCCESS) return fail(PYRO_ECUDA, "kernel launch: " + cu_err(r));
  }
  return PYRO_OK;
}
}  // namespace

int pyro_cn_step(const pyro_mech* hc, int64_t n, double dt, const double* rho, const double* T, const double* Y,
                 double tol, int max_newton, double* T_out, double* Y_out, int32_t* iters_out, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!rho || !T || !Y || !T_out || !Y_out)))
    return fail(PYRO_EINVAL, "pyro_cn_step: bad arguments");
  if (h && h->emitted.stats["jacobian_supported"] <= 0)
    return fail(PYRO_EINVAL, "the dense Jacobian kernels need all species to share one NASA-7 T_mid");
  if (!(dt >= 0.0) || !(tol > 0.0) || max_newton < 1 || max_newton > 1000)
    return fail(PYRO_EINVAL, "pyro_cn_step: need dt >= 0, tol > 0 and 1 <= max_newton <= 1000");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  if (int rc = ensure_groups(h, {"cn"})) return rc;
  const int64_t NS = h->m.n_species();
  const int refine = 1;
  if (int rc = cn_reserve(h, n)) return rc;
  int rc = with_args(h, n, {{rho, 1, 8, true, false}, {T, 1, 8, true, false}, {Y, NS, 8, true, false},
                            {T_out, 1, 8, false, true}, {Y_out, NS, 8, false, true}, {iters_out, 1, 4, false, true}},
                     stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                       return cn_run(h, nc, nc, dt, (const double*)d[0], (const double*)d[1], (const double*)d[2],
                                     tol, max_newton, refine, (double*)d[3], (double*)d[4], (int32_t*)d[5], st);
                     });
  if (rc) return rc;
  return maybe_checked(h, stream);
}

// ---- learned initial guess ---------------------------------------------------
namespace {
int ensure_mlp(pyro_mech* h) {
  if (h->emitted.stats["mlp_supported"] <= 0) return fail(PYRO_EINVAL, "the learned guess supports at most 63 species");
  if (!h->mlp) {
    if (int rc = pyro::mlp_create(h->m.n_species() + 1, &h->mlp)) return rc;
    if (cudaMalloc(&h->mlp_norm_dev, 4 * sizeof(float)) != cudaSuccess) return fail(PYRO_ECUDA, "MLP allocation");
  }
  return PYRO_OK;
}
int sync_norm(pyro_mech* h) {
  if (cudaMemcpy(h->mlp_norm_dev, pyro::mlp_host_norm(h->mlp), 4 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(PYRO_ECUDA, "MLP normalisation upload");
  return PYRO_OK;
}
}  // namespace

int pyro_mlp_n_params(const pyro_mech* h) { return h ? pyro::mlp_n_params(h->m.n_species() + 1) : 0; }

int pyro_mlp_set_params(pyro_mech* h, const double* params, const double* norm4) {
  if (!h || !params || !norm4) return fail(PYRO_EINVAL, "null argument");
  if (int rc = check_device(h)) return rc;
  if (int rc = ensure_mlp(h)) return rc;
  if (int rc = pyro::mlp_set(h->mlp, params, norm4)) return rc;
  return sync_norm(h);
}

int pyro_mlp_get_params(const pyro_mech* hc, double* params, double* norm4) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || !pyro::mlp_ready(h->mlp)) return fail(PYRO_ENOMLP, "no learned initial guess is loaded");
  return pyro::mlp_get(h->mlp, params, norm4);
}

int pyro_mlp_train(pyro_mech* h, int64_t n, const double* T, const double* Y, const char* options,
                   double* final_loss, void* stream) {
  if (!h || n <= 0 || !T || !Y) return fail(PYRO_EINVAL, "pyro_mlp_train: bad arguments");
  if (int rc = check_device(h)) return rc;
  if (classify({T, Y}) != 1) return fail(PYRO_EINVAL, "pyro_mlp_train takes device arrays");
  int epochs = 1, batch = 1024;
  double lr = 1e-2;
  unsigned seed = 1;
  if (options) {
    std::string str(options);
    for (char& c : str) if (c == ',') c = ';';
    std::stringstream ss(str);
    std::string kv;
    while (std::getline(ss, kv, ';')) {
      if (kv.empty()) continue;
      size_t eq = kv.find('=');
      if (eq == std::string::npos) return fail(PYRO_EINVAL, "option without '='");
      std::string k = kv.substr(0, eq), v = kv.substr(eq + 1);
      if (k == "epochs") epochs = std::atoi(v.c_str());
      else if (k == "batch") batch = std::atoi(v.c_str());
      else if (k == "lr") lr = std::atof(v.c_str());
      else if (k == "seed") seed = (unsigned)std::atol(v.c_str());
      else return fail(PYRO_EINVAL, "unknown training option '" + k + "'");
    }
  }
  if (epochs < 1 || batch < 64 || batch % 64 || !(lr > 0)) return fail(PYRO_EINVAL, "bad training options");
  if (int rc = ensure_mlp(h)) return rc;
  // internal energies of the training states by the library's energy kernel
  double* e = nullptr;
  if (cudaMalloc(&e, n * sizeof(double)) != cudaSuccess) return fail(PYRO_ECUDA, "training scratch allocation");
  int rc = pyro_internal_energy(h, n, T, Y, e, nullptr, stream);
  if (!rc) rc = pyro::mlp_train(h->mlp, n, h->m.n_species(), e, Y, T, epochs, batch, lr, seed, final_loss,
                                (cudaStream_t)stream);
  cudaFree(e);
  if (rc) return rc;
  return sync_norm(h);
}

int pyro_mlp_grad(const pyro_mech* hc, int64_t n, const double* e, const double* Y, const double* T,
                  double* loss, double* grad) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n <= 0 || n > (1 << 30) || !e || !Y || !T) return fail(PYRO_EINVAL, "pyro_mlp_grad: bad arguments");
  if (int rc = check_device(h)) return rc;
  if (!pyro::mlp_ready(h->mlp)) return fail(PYRO_ENOMLP, "no learned initial guess is loaded");
  if (classify({e, Y, T}) != 1) return fail(PYRO_EINVAL, "pyro_mlp_grad takes device arrays");
  return pyro::mlp_grad(h->mlp, n, 0, (int)n, h->m.n_species(), e, Y, T, loss, grad, 0);
}

int pyro_mlp_guess(const pyro_mech* hc, int64_t n, const double* e, const double* Y, double* y_out,
                   double* T_guess, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || (n > 0 && (!e || !Y || !y_out || !T_guess))) return fail(PYRO_EINVAL, "pyro_mlp_guess: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  if (!pyro::mlp_ready(h->mlp)) return fail(PYRO_ENOMLP, "no learned initial guess is loaded");
  const int64_t NS = h->m.n_species();
  return with_args(h, n, {{e, 1, 8, true, false}, {Y, NS, 8, true, false}, {y_out, 1, 8, false, true}, {T_guess, 1, 8, false, true}},
                   stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
                     long long nn = nc;
                     const void* wb = pyro::mlp_device_bf16(h->mlp);
                     const float* wf = pyro::mlp_device_params(h->mlp);
                     const float* nm = h->mlp_norm_dev;
                     void* pm[] = {&nn, &d[0], &d[1], &wb, &wf, &nm, &d[2], &d[3]};
                     return launch(h, h->f_mlp_guess, nc, 8, 0, st, pm);
                   });
}

int pyro_mlp_save(const pyro_mech* h, const char* path) {
  if (!h || !path) return fail(PYRO_EINVAL, "null argument");
  if (!pyro::mlp_ready(h->mlp)) return fail(PYRO_ENOMLP, "no learned initial guess is loaded");
  return pyro::mlp_save(h->mlp, path);
}

int pyro_mlp_load(pyro_mech* h, const char* path) {
  if (!h || !path) return fail(PYRO_EINVAL, "null argument");
  if (int rc = check_device(h)) return rc;
  if (int rc = ensure_mlp(h)) return rc;
  if (int rc = pyro::mlp_load(h->mlp, path)) return rc;
  return sync_norm(h);
}

int pyro_nonconverged(const pyro_mech* hc, void* stream, int64_t* count) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || !count) return fail(PYRO_EINVAL, "null argument");
  unsigned long long v = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&v, h->d_fail, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(h->d_fail, 0, sizeof v, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return fail(PYRO_ECUDA, "reading the failure counter");
  *count = (int64_t)v;
  return PYRO_OK;
}

int pyro_math_eval(const pyro_mech* hc, int fn, int64_t n, const double* x, double* y, void* stream) {
  pyro_mech* h = const_cast<pyro_mech*>(hc);
  if (!h || n < 0 || fn < 0 || fn > 2 || (n > 0 && (!x || !y))) return fail(PYRO_EINVAL, "pyro_math_eval: bad arguments");
  if (n == 0) return PYRO_OK;
  if (int rc = check_device(h)) return rc;
  return with_args(h, n, {{x, 1, 8, true, false}, {y, 1, 8, false, true}}, stream, [&](std::vector<void*>& d, int64_t nc, void* st) {
    long long nn = nc;
    void* params[] = {&fn, &nn, &d[0], &d[1]};
    return launch(h, h->f_math, nc, 8, 0, st, params);
  });
}

}  // extern "C"

// ---- internal helpers (not part of the C ABI) -------------------------------
#include "pyro_internal.h"

namespace pyro {

int internal_n_species(const pyro_mech* h) { return h ? h->m.n_species() : 0; }

int internal_check_device(const pyro_mech* h) {
  if (!h) return fail(PYRO_EINVAL, "null mechanism");
  return check_device(h);
}

int internal_fail(int code, const char* msg) { return fail(code, msg); }

int internal_launch_omega(const pyro_mech* h, int64_t n, const void* rho, const void* T_or_e,
                          int input_is_energy, const void* Y, void* T_out, void* omega,
                          unsigned long long* fail_ctr, void* stream) {
  long long nn = n;
  int em = input_is_energy ? 1 : 0;
  double Tg = 1200.0, tol = 1e-10;
  int max_iter = 50;
  void* store = h->d_store;
  void* params[] = {&nn, &rho, &T_or_e, &em, &Y, &T_out, &omega, &Tg, &max_iter, &tol, &fail_ctr, &store};
  // the same kernel choice as pyro_net_production_rates (thread or warp per state)
  if (h->opt.warp) {
    auto it = h->groups.find("wfwd");
    if (it == h->groups.end() || !it->second.f) return fail(PYRO_ECUDA, "warp-per-state kernel not loaded");
    return launch_warp(h, it->second, n, stream, params);
  }
  return launch(h, h->f_omega, n, h->omega_blocks_per_sm, h->emitted.smem_dyn_bytes_omega, stream, params);
}

}  // namespace pyro
