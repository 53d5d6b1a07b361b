// bst_multiply_execute_static: the native-FP64 split-K execute with its partial sums in
// a fixed, statically allocated device array instead of memory allocated at run time.
//
// Some callers cannot allocate device memory while they run: a service that reserves
// all of its GPU memory up front and forbids later cudaMalloc calls (an allocation can
// synchronise the device and stall every stream, which a latency-bound serving loop
// cannot accept), or a host framework that owns the whole device heap and has no way
// to hand out more.  For them this entry point takes the split-K workspace from
// g_splitk_scratch, a file-scope __device__ array that every GPU loading the library
// holds until the process exits.  The caller still passes the plan with its inputs and
// output bound; nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include <cmath>
#include <mutex>

#include "bst_internal.h"

namespace {

// 4 Mi doubles (32 MiB) per device.  Every call overwrites the whole region it uses
// (each (C block, part) writes all of its partial sums, zeros included), so nothing
// needs clearing between calls.
constexpr size_t kScratchDoubles = size_t(4) << 20;
static __device__ __align__(256) double g_splitk_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// The device address of g_splitk_scratch on the current device, looked up once per
// device (host code cannot take the array's address directly: the host-side symbol
// is only a stand-in).
double *scratch_address(int device) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_splitk_scratch);
    if (e != cudaSuccess || !p)
      throw bst::Error{BST_ERR_CUDA,
                       std::string("cudaGetSymbolAddress(g_splitk_scratch): ") + cudaGetErrorString(e)};
    g_addr[device] = static_cast<double *>(p);
  }
  return g_addr[device];
}

// Makes `device` current for the lifetime of the scope and then restores the device
// that was current before (only when they differ).
struct DeviceScope {
  int prev = -1;
  bool switched = false;
  explicit DeviceScope(int device) {
    BST_CUDA(cudaGetDevice(&prev));
    if (prev != device) {
      BST_CUDA(cudaSetDevice(device));
      switched = true;
    }
  }
  ~DeviceScope() {
    if (switched) (void)cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

size_t bst_static_scratch_doubles(void) { return kScratchDoubles; }

bst_status bst_multiply_execute_static(bst_plan *plan, double alpha, double beta, int32_t split_k,
                                       void *stream) {
  API_BEGIN
  BST_REQUIRE(plan, BST_ERR_INVALID_ARG, "plan is NULL");
  BST_REQUIRE(split_k >= 1 && split_k <= 64, BST_ERR_INVALID_ARG, "split_k must be in 1..64");
  BST_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), BST_ERR_INVALID_ARG,
              "alpha and beta must be finite");
  const int device = plan->ctx->device;
  BST_REQUIRE(device >= 0 && device < kMaxDevices, BST_ERR_UNSUPPORTED, "device index above 63");
  // every check that can fail comes before the first queued kernel: C_out's element
  // count is fixed by the plan, so the scratch bound is known here
  const bst_matrix *C = plan->C;
  const size_t need = (split_k > 1) ? (size_t)split_k * (size_t)C->nelem : 0;
  BST_REQUIRE(need <= kScratchDoubles, BST_ERR_UNSUPPORTED,
              "split_k x C elements = " + std::to_string(need) +
                  " doubles exceeds the static scratch of " + std::to_string(kScratchDoubles) +
                  " doubles; use bst_multiply_execute or a smaller split_k");
  const bool read_cin = beta != 0.0 && plan->Cin && plan->Cin->nblocks > 0;
  if (plan->contract) {
    bst::contract_check_bound(plan, read_cin);  // the tensors behind the matrix views
  } else {
    BST_REQUIRE(C->nelem == 0 || C->data, BST_ERR_STATE, "C_out data not bound");
    BST_REQUIRE(plan->A->nblocks == 0 || plan->A->data, BST_ERR_STATE, "A data not bound");
    BST_REQUIRE(plan->B->nblocks == 0 || plan->B->data, BST_ERR_STATE, "B data not bound");
    BST_REQUIRE(!read_cin || plan->Cin->data, BST_ERR_STATE, "C_in data not bound");
  }
  DeviceScope on(device);  // the caller's current device is restored on return
  double *W = scratch_address(device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (plan->contract) bst::contract_prepare(plan, read_cin, s);
  bst::NumArgs a;
  a.A = plan->A->data;
  a.B = plan->B->data;
  a.Cin = read_cin ? plan->Cin->data : nullptr;
  a.C = C->data;
  a.alpha = alpha;
  a.beta = read_cin ? beta : 0.0;
  bst::execute_fp64_workspace(plan, a, split_k, W, s);
  if (plan->contract) bst::contract_finish(plan, s);
  plan->stats.split_k = split_k;
  API_END
}

}  // extern "C"
