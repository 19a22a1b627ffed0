// K applied to spinors in device memory without allocating anything at call time.
//
// The ordinary entry point ovl_wilson_apply converts the caller's canonical spinors
// into the library's chunked layout in workspaces that it allocates on demand. Some
// callers cannot let a library allocate while they run: code that has handed all
// device memory to its own pool or runs under a hard memory cap, and real-time loops
// that must not stall on the allocator. For them this variant keeps the two
// layout-conversion buffers in one file-scope __device__ array instead.
//
// The array (OVL_NOALLOC_BYTES) exists once per device that loads the library and
// stays allocated until the process exits. Host code cannot use its name as an
// address (on the host the symbol is only a stand-in); its device address is looked up
// once per device with cudaGetSymbolAddress on the first call made on that device
// and cached; that first call belongs before any stream capture begins. Every call shares the array: calls that overlap on the GPU (other
// streams, other host threads) race on it, and after a call it holds that call's
// intermediate fields. Nothing in it needs to start at zero, because each call writes
// every byte it later reads.
#include <mutex>

#include "context.h"

namespace ovl {

constexpr size_t kNoAllocBytes = OVL_NOALLOC_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256] = {nullptr};

static ovl_status noalloc_base(ovl_ctx* c, void** out) {
  int dev = 0;
  OVL_CUDA(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_err(c, OVL_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaGetSymbolAddress(static scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return OVL_OK;
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_wilson_apply_noalloc(ovl_ctx* c, const void* in, void* out, int n, int dtype, int prec) {
  if (!c) return OVL_EINVAL;
  if (!in || !out) return set_err(c, OVL_EINVAL, "null spinor pointer");
  if (n < 1) return set_err(c, OVL_EINVAL, "n must be >= 1");
  if (dtype != OVL_C128 && dtype != OVL_C64) return set_err(c, OVL_EINVAL, "dtype must be OVL_C128 or OVL_C64");
  if (prec < P64 || prec > P16) return set_err(c, OVL_EINVAL, "prec must be OVL_PREC_F64, F32 or F16");
  int dev = -1;
  OVL_CUDA(c, cudaGetDevice(&dev));
  if (dev != c->device) return set_err(c, OVL_EINVAL, "the context's device must be current");
  const size_t per = (size_t)c->V * spinor_site_bytes(prec);
  const size_t field = round256(per * n);
  const size_t norms = prec == P16 ? round256(sizeof(float) * c->V * (size_t)n) : 0;
  const size_t need = 2 * (field + norms);
  if (need > kNoAllocBytes) {
    char m[200];
    snprintf(m, sizeof(m), "n * V = %lld needs %zu bytes of static scratch, more than the %zu available",
             (long long)n * c->V, need, kNoAllocBytes);
    return set_err(c, OVL_EINVAL, m);
  }
  void* base = nullptr;
  OVL_TRY(noalloc_base(c, &base));
  char* b = static_cast<char*>(base);
  Field fin, fout;
  fin.prec = fout.prec = prec;
  fin.n = fout.n = n;
  fin.V = fout.V = c->V;
  fin.data = b;
  fout.data = b + field;
  if (prec == P16) {
    fin.norm = reinterpret_cast<float*>(b + 2 * field);
    fout.norm = reinterpret_cast<float*>(b + 2 * field + norms);
  }
  launch_pack(dtype, in, prec, fin.ref(), n, c->V, c->st);
  launch_wilson_K(prec, prec, prec, c->g, c->kappa, links_of(c, prec), fin.ref(), fout.ref(), n, nullptr, nullptr,
                  c->st);
  launch_unpack(dtype, out, prec, fout.ref(), n, c->V, c->st);
  OVL_TRY(check_launch(c, __func__));
  OVL_CUDA(c, cudaStreamSynchronize(c->st));
  return OVL_OK;
}
