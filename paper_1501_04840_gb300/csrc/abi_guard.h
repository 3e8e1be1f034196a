// Exception barrier of the C ABI: an entry point runs its body through ot_guard, so
// that a C++ exception (a failed host allocation in a table or staging vector, say)
// becomes a status and a message for ot_last_error instead of crossing the C boundary.
#pragma once
#include <exception>
#include <new>

#include "../../include/dynot.h"

namespace dynot {

ot_status seterr(ot_status s, const char* fmt, ...);

template <class F>
ot_status ot_guard(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return seterr(OT_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return seterr(OT_ECUDA, "internal error: %s", e.what());
  } catch (...) {
    return seterr(OT_ECUDA, "internal error");
  }
}

}  // namespace dynot
