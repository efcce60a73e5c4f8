// Allocation-failure injection for tests (dos_test_fail_alloc): every device
// allocation the library makes asks this first, so a test can make any one
// of them fail exactly as an out-of-memory cudaMalloc would and check that
// the call reports DOS_ENOMEM, releases what it had taken and leaves the
// library usable.  Disarmed (the default) it costs one atomic load.
#pragma once

namespace netdos {

// true when this allocation is the one the armed hook makes fail (the hook
// then disarms itself)
bool alloc_fault_injected();

}  // namespace netdos
