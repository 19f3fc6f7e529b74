// Host-side fault injection for tests of failure handling. With the environment variable
// HYGRO_FAULT=<entry point>:<n>, the n-th call (counted from 1 in the process) of the named C-ABI entry
// point fails with HYGRO_E_CUDA before it changes anything or touches the device. Nothing here makes a
// device fault, trap or hang. Plain C++ without CUDA: the library (hygro_api.cu) includes it, and the CPU
// tests compile it on their own.
#pragma once

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

namespace hygro {

struct FaultSpec {
    char call[64];
    int64_t n;      // the call to fail, counted from 1
    bool active;
};

// "<name>:<n>" with a non-empty name of at most 63 characters and n >= 1; anything else is inactive.
inline FaultSpec parse_fault(const char *spec)
{
    FaultSpec f;
    memset(&f, 0, sizeof f);
    if (spec == nullptr) return f;
    const char *colon = strrchr(spec, ':');
    if (colon == nullptr || colon == spec || colon - spec >= (ptrdiff_t)sizeof f.call) return f;
    char *end = nullptr;
    const long long n = strtoll(colon + 1, &end, 10);
    if (end == colon + 1 || *end != '\0' || n < 1) return f;
    memcpy(f.call, spec, (size_t)(colon - spec));
    f.call[colon - spec] = '\0';
    f.n = n;
    f.active = true;
    return f;
}

// Counts the calls of the named entry point and says which one is to fail.
class FaultInjector {
  public:
    explicit FaultInjector(const FaultSpec &s) : spec_(s) {}
    bool hit(const char *call)
    {
        if (!spec_.active || strcmp(call, spec_.call) != 0) return false;
        std::lock_guard<std::mutex> lock(m_);
        return ++count_ == spec_.n;
    }

  private:
    FaultSpec spec_;
    int64_t count_ = 0;
    std::mutex m_;
};

}  // namespace hygro
