// Library-owned CUDA objects (streams, events) cached per CUDA context.  An entry is keyed on
// the device and the unique id of the context current when it was made.  A device reset
// destroys the primary context with every stream and event in it, and their handles may later
// name objects the caller creates; the next call runs in a new context, with a new id, and so
// makes fresh objects instead of using the stale handles.  Objects of a destroyed context are
// not released (their handles are no longer valid).  With more than N live (context, device)
// pairs the oldest entry is reused and its objects are left alive.  Plain C++: the CUDA calls
// are in the caller's make function.
#pragma once

namespace skel {

template <typename T, int N = 64>
class ContextCache {
 public:
  // The entry of (ctx, dev), made by make(T&) -> bool on first use; nullptr when make fails,
  // and nothing is cached then.  The caller serialises get() and every use of the result.
  template <typename Make>
  T* get(unsigned long long ctx, int dev, Make&& make) {
    for (int i = 0; i < N; ++i)
      if (used_[i] && ctx_[i] == ctx && dev_[i] == dev) return &val_[i];
    T fresh{};
    if (!make(fresh)) return nullptr;
    const int i = next_;
    next_ = (next_ + 1) % N;
    val_[i] = fresh;
    ctx_[i] = ctx;
    dev_[i] = dev;
    used_[i] = true;
    return &val_[i];
  }

 private:
  T val_[N] = {};
  unsigned long long ctx_[N] = {};
  int dev_[N] = {};
  bool used_[N] = {};
  int next_ = 0;
};

}  // namespace skel
