// Host-side fault injection (tnc_inject_failure): makes one chosen call site
// of the library fail on the host, so that callers' error handling (and the
// library's own all-or-nothing cleanup) can be exercised without any device
// fault.  Process-wide: one armed failure at a time.
#include <atomic>
#include <mutex>

#include "tnc_internal.h"

namespace {
std::mutex g_mu;
int g_kind = TNC_INJECT_NONE;
int g_after = 0;
std::atomic<int> g_armed{0};
}  // namespace

namespace tnc {

bool inject_hit(int kind) {
  if (!g_armed.load(std::memory_order_relaxed)) return false;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_kind != kind) return false;
  if (g_after > 0) {
    g_after--;
    return false;
  }
  g_kind = TNC_INJECT_NONE;
  g_armed.store(0);
  return true;
}

}  // namespace tnc

extern "C" int tnc_inject_failure(int32_t kind, int32_t after) {
  tnc::clear_error();
  if (kind < TNC_INJECT_NONE || kind > TNC_INJECT_TIMEOUT || after < 0)
    return tnc::set_error(TNC_ERR_INVALID, "unknown injection kind or negative count");
  std::lock_guard<std::mutex> lock(g_mu);
  g_kind = kind;
  g_after = after;
  g_armed.store(kind != TNC_INJECT_NONE ? 1 : 0);
  return TNC_OK;
}
