// Run-time specialisation of the standard FP32 step kernels: the plane wave
// (table and learned samplers) and the Yee grid (plain gather and the
// tile-staged kernel).
//
// The kernel source of push_emit.cu (embedded in the library at build time)
// is compiled by NVRTC with -DPRAD_SPEC and the context's per-run constants
// as literals (spec_params in push_emit.cu), loaded with the driver API and
// launched in place of the ahead-of-time instantiation.  The constants are
// the values the host would otherwise pass in StepParams, printed exactly
// (hexadecimal floating point), so the specialised kernel computes the same
// bits; it only saves their loads and lets them fold into the arithmetic.
//
// NVRTC is opened with dlopen when the first kernel is wanted, so the
// library loads without it; driver functions come from the runtime's
// entry-point query (no link against libcuda).
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "prad_internal.h"

// kSpecSrcName / kSpecSrc: the kernel translation unit and the headers it
// includes, written by the build script
#include "prad_spec_sources.inc"

#ifndef PRAD_CUDA_INCLUDE
#define PRAD_CUDA_INCLUDE "/usr/local/cuda/include"
#endif
#ifndef PRAD_CUDA_LIBDIR
#define PRAD_CUDA_LIBDIR "/usr/local/cuda/lib64"
#endif

namespace prad {
namespace {

// ---- NVRTC, opened on first use ---------------------------------------------
struct Nvrtc {
  bool ok = false;
  std::string why;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) err_str = nullptr;
};

// ---- driver functions, from the runtime's entry-point query -----------------
struct Driver {
  bool ok = false;
  std::string why;
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleUnload) unload = nullptr;
  decltype(&cuModuleGetFunction) get_function = nullptr;
  decltype(&cuLaunchKernel) launch = nullptr;
  decltype(&cuOccupancyMaxActiveBlocksPerMultiprocessor) occupancy = nullptr;
  decltype(&cuCtxGetCurrent) ctx_current = nullptr;
  decltype(&cuFuncSetAttribute) set_attr = nullptr;
};

template <class F>
bool sym(void* h, const char* name, F* out) {
  *out = reinterpret_cast<F>(dlsym(h, name));
  return *out != nullptr;
}

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    // PRAD_NVRTC_LIBRARY names the NVRTC library to open instead of the
    // toolkit's (and only it)
    const char* lib = std::getenv("PRAD_NVRTC_LIBRARY");
    void* h = nullptr;
    if (lib && *lib) {
      h = dlopen(lib, RTLD_NOW | RTLD_LOCAL);
    } else {
      h = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
      if (!h) h = dlopen(PRAD_CUDA_LIBDIR "/libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
      if (!h) h = dlopen("libnvrtc.so", RTLD_NOW | RTLD_LOCAL);
    }
    if (!h) {
      const char* e = dlerror();
      n.why = std::string("cannot open NVRTC: ") + (e ? e : "libnvrtc.so.13 not found");
      return;
    }
    n.ok = sym(h, "nvrtcCreateProgram", &n.create) && sym(h, "nvrtcAddNameExpression", &n.add_name) &&
           sym(h, "nvrtcCompileProgram", &n.compile) &&
           sym(h, "nvrtcGetProgramLogSize", &n.log_size) && sym(h, "nvrtcGetProgramLog", &n.log) &&
           sym(h, "nvrtcGetCUBINSize", &n.cubin_size) && sym(h, "nvrtcGetCUBIN", &n.cubin) &&
           sym(h, "nvrtcGetLoweredName", &n.lowered) && sym(h, "nvrtcDestroyProgram", &n.destroy) &&
           sym(h, "nvrtcGetErrorString", &n.err_str);
    if (!n.ok) n.why = "NVRTC library lacks an expected symbol";
  });
  return n;
}

template <class F>
bool entry(const char* name, F* out) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *out = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    d.ok = entry("cuModuleLoadData", &d.load) && entry("cuModuleUnload", &d.unload) &&
           entry("cuModuleGetFunction", &d.get_function) && entry("cuLaunchKernel", &d.launch) &&
           entry("cuOccupancyMaxActiveBlocksPerMultiprocessor", &d.occupancy) &&
           entry("cuCtxGetCurrent", &d.ctx_current) &&
           entry("cuFuncSetAttribute", &d.set_attr);
    if (!d.ok) d.why = "driver entry points unavailable";
  });
  return d;
}

// The constants a specialised kernel has compiled in, with its variant.
struct SpecKey {
  float half_q_dtn, dtn, inv_dtn, cn_dt, eps_r15, ll_coef, E0, kc, kc_lo, cp_dt;
  float inv_dx, inv_dy, inv_dx_lo, inv_dy_lo, x0, y0, Lx, Ly;  // Yee grid
  int32_t nx, ny, ntx;
  uint64_t phase_step;
  uint32_t ensemble;
  uint32_t rkey[20];
  SpecVariant v;
};

SpecKey key_of(const StepParams<float>& p, const SpecVariant& v) {
  SpecKey k;
  std::memset(&k, 0, sizeof(k));
  k.half_q_dtn = p.half_q_dtn;
  k.dtn = p.dtn;
  k.inv_dtn = p.inv_dtn;
  k.cn_dt = p.cn_dt;
  k.eps_r15 = p.eps_r15;
  k.ll_coef = p.ll_coef;
  k.E0 = p.E0;
  k.kc = p.kc;
  k.kc_lo = p.kc_lo;
  k.cp_dt = p.cp_dt;
  if (v.field == PRAD_FIELD_YEE2D) {
    k.inv_dx = p.inv_dx;
    k.inv_dy = p.inv_dy;
    k.inv_dx_lo = p.inv_dx_lo;
    k.inv_dy_lo = p.inv_dy_lo;
    k.x0 = p.x0;
    k.y0 = p.y0;
    k.Lx = p.Lx;
    k.Ly = p.Ly;
    k.nx = p.nx;
    k.ny = p.ny;
    k.ntx = v.tiled ? p.ntx : 0;
  }
  k.phase_step = p.phase_step;
  k.ensemble = p.ensemble;
  std::memcpy(k.rkey, p.rkey, sizeof(k.rkey));
  k.v = v;
  return k;
}

bool same(const SpecKey& a, const SpecKey& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

// -D options carrying the constants: floats as exact hexadecimal literals
bool spec_defines(const SpecKey& k, std::vector<std::string>& out) {
  const float v[10] = {k.half_q_dtn, k.dtn, k.inv_dtn, k.cn_dt, k.eps_r15,
                       k.ll_coef,    k.E0,  k.kc,      k.kc_lo, k.cp_dt};
  const char* nm[10] = {"HALF_Q_DTN", "DTN", "INV_DTN", "CN_DT", "EPS_R15",
                        "LL_COEF",    "E0",  "KC",      "KC_LO", "CP_DT"};
  char buf[512];
  for (int j = 0; j < 10; ++j) {
    if (!std::isfinite(v[j])) return false;
    std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_%s=(%af)", nm[j], static_cast<double>(v[j]));
    out.emplace_back(buf);
  }
  std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_PHASE_STEP=%lluull",
                static_cast<unsigned long long>(k.phase_step));
  out.emplace_back(buf);
  std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_ENSEMBLE=%uu", k.ensemble);
  out.emplace_back(buf);
  std::string rk = "-DPRAD_SPEC_RKEY={";
  for (int j = 0; j < 20; ++j) {
    std::snprintf(buf, sizeof(buf), "%uu%s", k.rkey[j], j < 19 ? "," : "}");
    rk += buf;
  }
  out.push_back(rk);
  if (k.v.field == PRAD_FIELD_YEE2D) {
    const float y[8] = {k.inv_dx, k.inv_dy, k.inv_dx_lo, k.inv_dy_lo, k.x0, k.y0, k.Lx, k.Ly};
    const char* ynm[8] = {"INV_DX", "INV_DY", "INV_DX_LO", "INV_DY_LO", "X0", "Y0", "LX", "LY"};
    for (int j = 0; j < 8; ++j) {
      if (!std::isfinite(y[j])) return false;
      std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_%s=(%af)", ynm[j], static_cast<double>(y[j]));
      out.emplace_back(buf);
    }
    std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_NX=%d", k.nx);
    out.emplace_back(buf);
    std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_NY=%d", k.ny);
    out.emplace_back(buf);
    std::snprintf(buf, sizeof(buf), "-DPRAD_SPEC_NTX=%d", k.ntx);
    out.emplace_back(buf);
    out.emplace_back("-DPRAD_SPEC_YEE");
  }
  return true;
}

std::string cuda_include() {
  const char* home = std::getenv("CUDA_HOME");
  if (home && *home) return std::string(home) + "/include";
  return PRAD_CUDA_INCLUDE;
}

}  // namespace

struct SpecFn {
  SpecKey key;
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
  CUcontext ctx = nullptr;
  int device = 0;
  unsigned dyn_smem = 0;  // dynamic shared memory per block
};

struct SpecCache {
  std::vector<SpecFn*> fns;
};

SpecCache* spec_create() { return new SpecCache(); }

void spec_destroy(SpecCache* c) {
  if (!c) return;
  const Driver& d = driver();
  for (SpecFn* f : c->fns) {
    if (d.ok && f->mod) d.unload(f->mod);
    delete f;
  }
  delete c;
}

namespace {
cudaError_t spec_get_impl(SpecCache* c, int device, const StepParams<float>& p,
                          const SpecVariant& v, const SpecFn** out, std::string* msg) {
  const SpecKey key = key_of(p, v);
  for (SpecFn* f : c->fns)
    if (same(f->key, key)) {
      *out = f;
      return cudaSuccess;
    }
  const Nvrtc& nv = nvrtc();
  if (!nv.ok) {
    *msg = nv.why;
    return cudaErrorNotSupported;
  }
  const Driver& d = driver();
  if (!d.ok) {
    *msg = d.why;
    return cudaErrorNotSupported;
  }
  // the ahead-of-time build's code-generation defaults (FMA contraction on,
  // IEEE division and square root, no flush to zero) are NVRTC's too
  std::vector<std::string> opts = {"-arch=sm_103a", "-std=c++17", "-default-device",
                                   "-DPRAD_SPEC", "-I" + cuda_include()};
  if (!spec_defines(key, opts)) {
    *msg = "run-time specialisation: non-finite constant";
    return cudaErrorInvalidValue;
  }
  char name[160];
  if (v.tiled)
    std::snprintf(name, sizeof(name), "prad::k_push_emit_tiled<float, false, true>");
  else
    std::snprintf(name, sizeof(name), "prad::k_push_emit<float, %d, %d, %d, false, true, %d>",
                  v.field, v.samp, v.pf, v.pws);
  constexpr int kNSrc = sizeof(kSpecSrc) / sizeof(kSpecSrc[0]);
  nvrtcProgram prog = nullptr;
  if (nv.create(&prog, kSpecSrc[0], kSpecSrcName[0], kNSrc - 1, kSpecSrc + 1, kSpecSrcName + 1) !=
      NVRTC_SUCCESS) {
    *msg = "nvrtcCreateProgram failed";
    return cudaErrorUnknown;
  }
  std::vector<const char*> argv;
  for (const std::string& o : opts) argv.push_back(o.c_str());
  nv.add_name(prog, name);
  const nvrtcResult r = nv.compile(prog, static_cast<int>(argv.size()), argv.data());
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nv.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) nv.log(prog, &log[0]);
    *msg = std::string("NVRTC: ") + nv.err_str(r) + ": " + log.substr(0, 400);
    nv.destroy(&prog);
    return cudaErrorUnknown;
  }
  size_t nbin = 0;
  nv.cubin_size(prog, &nbin);
  std::vector<char> bin(nbin);
  nv.cubin(prog, bin.data());
  const char* lowered = nullptr;
  nv.lowered(prog, name, &lowered);
  const std::string sym_name = lowered ? lowered : "";
  nv.destroy(&prog);
  // the runtime makes the device's primary context current on this thread;
  // the thread's current device is put back on return
  struct DeviceGuard {
    int prev = -1;
    ~DeviceGuard() {
      int now = -1;
      if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
  } guard;
  if (cudaGetDevice(&guard.prev) != cudaSuccess) guard.prev = -1;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return e;
  SpecFn* f = new SpecFn();
  f->key = key;
  f->device = device;
  CUresult cr = d.ctx_current(&f->ctx);
  if (cr == CUDA_SUCCESS) cr = d.load(&f->mod, bin.data());
  if (cr == CUDA_SUCCESS) cr = d.get_function(&f->fn, f->mod, sym_name.c_str());
  if (cr == CUDA_SUCCESS && v.tiled) {
    // the staged field tile (dynamic) and the photon stage exceed 48 KB
    f->dyn_smem = kTileSmemBytes;
    cr = d.set_attr(f->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, kTileSmemBytes);
  }
  if (cr != CUDA_SUCCESS) {
    if (f->mod) d.unload(f->mod);
    delete f;
    char b[96];
    std::snprintf(b, sizeof(b), "loading the specialised kernel failed (CUresult %d)",
                  static_cast<int>(cr));
    *msg = b;
    return cudaErrorUnknown;
  }
  c->fns.push_back(f);
  *out = f;
  return cudaSuccess;
}
}  // namespace

cudaError_t spec_get(SpecCache* c, int device, const StepParams<float>& p, const SpecVariant& v,
                     const SpecFn** out, char* msg, size_t msg_len) {
  *out = nullptr;
  std::string m;
  const cudaError_t e = spec_get_impl(c, device, p, v, out, &m);
  if (e != cudaSuccess && msg && msg_len) std::snprintf(msg, msg_len, "%s", m.c_str());
  return e;
}

int spec_occupancy(const SpecFn* f, int block) {
  int nb = 0;
  if (driver().occupancy(&nb, f->fn, block, f->dyn_smem) != CUDA_SUCCESS) return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t spec_launch(const SpecFn* f, const StepParams<float>& p, int grid, int block,
                        cudaStream_t s) {
  const Driver& d = driver();
  CUcontext cur = nullptr;
  int prev = -1;
  if (d.ctx_current(&cur) != CUDA_SUCCESS || cur != f->ctx) {
    // another device (or none) current on this thread: bind the kernel's
    // for the launch and put the thread's device back after it
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    const cudaError_t e = cudaSetDevice(f->device);
    if (e != cudaSuccess) return e;
    if (d.ctx_current(&cur) != CUDA_SUCCESS || cur != f->ctx) return cudaErrorInvalidResourceHandle;
  }
  void* args[] = {const_cast<StepParams<float>*>(&p)};
  const CUresult r = d.launch(f->fn, static_cast<unsigned>(grid), 1, 1, static_cast<unsigned>(block),
                              1, 1, f->dyn_smem, reinterpret_cast<CUstream>(s), args, nullptr);
  if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
  switch (r) {
    case CUDA_SUCCESS: return cudaSuccess;
    case CUDA_ERROR_INVALID_VALUE: return cudaErrorInvalidValue;
    case CUDA_ERROR_INVALID_HANDLE: return cudaErrorInvalidResourceHandle;
    case CUDA_ERROR_LAUNCH_OUT_OF_RESOURCES: return cudaErrorLaunchOutOfResources;
    default: return cudaErrorLaunchFailure;
  }
}

}  // namespace prad
