// Model-specialised builds of the batched kernels, compiled at run time.
//
// The batched kernels read a model's counts and scratch offsets (DevModel's
// integer fields) and the launch shape (team size, dense row capacity, scratch
// stride) from memory; every scratch access then costs a load of its offset and
// the address arithmetic around it.  For one model and one launch shape those
// values are constants: this file writes them into the kernels' source as
// literals (every `M.<field>` of the device code becomes a number; the launch
// shape comes in through the SHAC_SPEC_* macros of shac_batched.cuh, the link
// parents through SHAC_SPEC_PARENTS of shac_device.cuh), compiles
// the forward and adjoint kernels with NVRTC for the device's architecture and
// loads them with the runtime's library API.  The sources are the library's
// own device files, embedded at build time (shac_jit_sources.cpp, written by
// build.py).  Builds are cached for the life of the process, per device, model
// layout and launch shape.
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <regex>
#include <string>
#include <vector>

#include "shac_jit.h"

extern const char* const shac_jit_src_device;    // shac_device.cuh
extern const char* const shac_jit_src_kernels;   // shac_kernels.cuh
extern const char* const shac_jit_src_batched;   // shac_batched.cuh

namespace shac {
namespace {

struct Field {
  const char* name;
  int DevModel::*member;
};

// Every integer field of DevModel: counts, flags and scratch offsets.
const Field kFields[] = {
    {"L", &DevModel::L}, {"nq", &DevModel::nq}, {"nv", &DevModel::nv}, {"na", &DevModel::na},
    {"ntact", &DevModel::ntact}, {"nc", &DevModel::nc}, {"nm", &DevModel::nm}, {"nseg", &DevModel::nseg},
    {"nitems", &DevModel::nitems}, {"K", &DevModel::K}, {"nlev", &DevModel::nlev},
    {"root_free", &DevModel::root_free}, {"height_q", &DevModel::height_q}, {"vx_dof", &DevModel::vx_dof},
    {"o_Q", &DevModel::o_Q}, {"o_QD", &DevModel::o_QD}, {"o_ACT", &DevModel::o_ACT}, {"o_QB", &DevModel::o_QB},
    {"o_QDB", &DevModel::o_QDB}, {"o_ACTB", &DevModel::o_ACTB}, {"o_LR", &DevModel::o_LR},
    {"o_LW", &DevModel::o_LW}, {"o_S", &DevModel::o_S}, {"o_IT", &DevModel::o_IT}, {"o_M", &DevModel::o_M},
    {"o_LD", &DevModel::o_LD}, {"o_B", &DevModel::o_B}, {"o_T", &DevModel::o_T}, {"o_QDD", &DevModel::o_QDD},
    {"o_QC", &DevModel::o_QC}, {"o_QDC", &DevModel::o_QDC}, {"o_LAM", &DevModel::o_LAM},
    {"o_ITB", &DevModel::o_ITB}, {"o_SEGA", &DevModel::o_SEGA}, {"o_MW", &DevModel::o_MW},
    {"o_RDB", &DevModel::o_RDB}, {"rec_floats", &DevModel::rec_floats}, {"env_floats", &DevModel::env_floats},
};

// Replace every `M.<field>` (as a whole word) by the field's value.
std::string with_literals(const char* src, const DevModel& m) {
  std::string s(src);
  for (const Field& f : kFields) {
    const std::regex re(std::string("\\bM\\.") + f.name + "\\b");
    s = std::regex_replace(s, re, "(" + std::to_string(m.*(f.member)) + ")");
  }
  return s;
}

// the parent list as a C initialiser list ("-1,0,0,1")
std::string parent_list(const std::vector<int>& parent) {
  std::string s;
  for (size_t i = 0; i < parent.size(); ++i) s += (i ? "," : "") + std::to_string(parent[i]);
  return s;
}

std::string spec_string(int device, const DevModel& m, const std::vector<int>& parent, int lanes, int rows,
                        int stride) {
  std::string s = "dev" + std::to_string(device) + ";lanes" + std::to_string(lanes) + ";rows" +
                  std::to_string(rows) + ";stride" + std::to_string(stride);
  for (const Field& f : kFields) s += ";" + std::string(f.name) + "=" + std::to_string(m.*(f.member));
  return s + ";parents=" + parent_list(parent);
}

// FNV-1a; 0 is reserved for the generic kernels
unsigned int key_of(const std::string& s) {
  unsigned int h = 2166136261u;
  for (unsigned char c : s) { h ^= c; h *= 16777619u; }
  return h == 0u ? 1u : h;
}

std::mutex g_mutex;
std::map<std::string, JitKernels> g_cache;

}  // namespace

shac_status jit_kernels(int device, const DevModel& m, const std::vector<int>& parent, int lanes, int rows,
                        int stride, JitKernels* out, std::string* log) {
  if ((int)parent.size() != m.L) return SHAC_ERR_INVALID_ARG;
  const std::string spec = spec_string(device, m, parent, lanes, rows, stride);
  std::lock_guard<std::mutex> lock(g_mutex);
  auto it = g_cache.find(spec);
  if (it != g_cache.end()) { *out = it->second; return SHAC_OK; }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess)
    return SHAC_ERR_CUDA;
  const unsigned int key = key_of(spec);
  const std::string h_device = with_literals(shac_jit_src_device, m);
  const std::string h_kernels = with_literals(shac_jit_src_kernels, m);
  const std::string h_batched = with_literals(shac_jit_src_batched, m);
  const char* headers[] = {h_device.c_str(), h_kernels.c_str(), h_batched.c_str()};
  const char* names[] = {"shac_device.cuh", "shac_kernels.cuh", "shac_batched.cuh"};
  const char* main_src =
      "#include \"shac_batched.cuh\"\n"
      "template __global__ void shac::k_batched<false>(shac::BatchedArgs);\n"
      "template __global__ void shac::k_batched<true>(shac::BatchedArgs);\n";
  nvrtcProgram prog = nullptr;
  if (nvrtcCreateProgram(&prog, main_src, "shac_batched_spec.cu", 3, headers, names) != NVRTC_SUCCESS)
    return SHAC_ERR_CUDA;
  nvrtcAddNameExpression(prog, "shac::k_batched<false>");
  nvrtcAddNameExpression(prog, "shac::k_batched<true>");
  const std::string arch = "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor) + "a";
  char kbuf[64], lbuf[64], rbuf[64], sbuf[64];
  std::snprintf(kbuf, sizeof kbuf, "-DSHAC_SPEC_KEY=%uu", key);
  std::snprintf(lbuf, sizeof lbuf, "-DSHAC_SPEC_LANES=%d", lanes);
  std::snprintf(rbuf, sizeof rbuf, "-DSHAC_SPEC_ROWS=%d", rows);
  std::snprintf(sbuf, sizeof sbuf, "-DSHAC_SPEC_STRIDE=%d", stride);
  const std::string pdef = "-DSHAC_SPEC_PARENTS=" + parent_list(parent);
  const char* opts[] = {arch.c_str(), "-std=c++17", "-lineinfo", kbuf, lbuf, rbuf, sbuf, pdef.c_str()};
  const nvrtcResult cr = nvrtcCompileProgram(prog, (int)(sizeof opts / sizeof opts[0]), opts);
  if (cr != NVRTC_SUCCESS) {
    if (log) {
      size_t n = 0;
      nvrtcGetProgramLogSize(prog, &n);
      std::vector<char> buf(n + 1, 0);
      nvrtcGetProgramLog(prog, buf.data());
      *log = buf.data();
    }
    nvrtcDestroyProgram(&prog);
    return SHAC_ERR_CUDA;
  }
  const char* lowered[2] = {nullptr, nullptr};
  size_t cubin_size = 0;
  if (nvrtcGetLoweredName(prog, "shac::k_batched<false>", &lowered[0]) != NVRTC_SUCCESS ||
      nvrtcGetLoweredName(prog, "shac::k_batched<true>", &lowered[1]) != NVRTC_SUCCESS ||
      nvrtcGetCUBINSize(prog, &cubin_size) != NVRTC_SUCCESS || cubin_size == 0) {
    nvrtcDestroyProgram(&prog);
    return SHAC_ERR_CUDA;
  }
  std::vector<char> cubin(cubin_size);
  const std::string name_fwd = lowered[0], name_adj = lowered[1];
  const bool got = nvrtcGetCUBIN(prog, cubin.data()) == NVRTC_SUCCESS;
  nvrtcDestroyProgram(&prog);
  if (!got) return SHAC_ERR_CUDA;
  JitKernels k;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kf = nullptr, ka = nullptr;
  if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&kf, lib, name_fwd.c_str()) != cudaSuccess ||
      cudaLibraryGetKernel(&ka, lib, name_adj.c_str()) != cudaSuccess)
    return SHAC_ERR_CUDA;
  k.fwd = reinterpret_cast<const void*>(kf);
  k.adj = reinterpret_cast<const void*>(ka);
  k.key = key;
  g_cache[spec] = k;
  *out = k;
  return SHAC_OK;
}

}  // namespace shac
