// faults.cu -- host-side fault injection for failure tests (the paper has no
// counterpart).  A fault is armed by the INPC_FAULT environment variable
// (read once, at the library's first use) or by inpc_set_fault; nothing is
// ever injected on the device, and no fault makes a GPU trap or hang.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"

namespace inpc {
namespace {

std::mutex g_fault_mu;
bool g_env_read = false;
std::string g_fault;  // armed fault spec ("" = none)

void read_env_locked() {
  if (g_env_read) return;
  g_env_read = true;
  const char* e = std::getenv("INPC_FAULT");
  if (e) g_fault = e;
}

bool armed(const char* name) {
  std::lock_guard<std::mutex> lk(g_fault_mu);
  read_env_locked();
  return g_fault == name;
}

}  // namespace

bool fault_workspace_overflow() { return armed("workspace_overflow"); }

bool fault_corrupt_args() { return armed("corrupt_args"); }

uint32_t fault_take_queue_short() {
  std::lock_guard<std::mutex> lk(g_fault_mu);
  read_env_locked();
  if (g_fault != "queue_short") return 0;
  g_fault.clear();  // one launch only
  return 1;
}

}  // namespace inpc

extern "C" inpc_status inpc_set_fault(const char* spec) {
  using namespace inpc;
  static const char* known[] = {"workspace_overflow", "corrupt_args", "queue_short"};
  std::string s = spec ? spec : "";
  if (!s.empty()) {
    bool ok = false;
    for (const char* k : known) ok = ok || s == k;
    if (!ok) return fail(INPC_ERR_INVALID_ARG, "inpc_set_fault: unknown fault '%s'", s.c_str());
  }
  std::lock_guard<std::mutex> lk(g_fault_mu);
  g_env_read = true;  // an explicit setting replaces the environment's
  g_fault = s;
  return INPC_OK;
}
