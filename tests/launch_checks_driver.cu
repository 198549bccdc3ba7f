// Host-side checks of the launch-check registry (no GPU: without a device the
// registry keys every entry by the same device, -1). Built and run by
// tests/test_launch_checks.py against the library's own prof.cu.
#include <cstdio>
#include <string>
#include <thread>
#include "gcp_internal.cuh"
using namespace gcp;
int main() {
  alignas(256) static unsigned char lib[4096];
  const void* B = lib;
  reg_alloc(B, 1024);
  int fails = 0;
  auto expect = [&](bool got, bool want, const char* what) {
    if (got != want) { std::printf("FAIL %s\n", what); ++fails; }
  };
  const uint64_t t = reg_foreign(B, 64);
  expect(reg_check(B, 512, "a"), true, "library entry covers with a foreign one at the same base");
  reg_unforeign(t);
  expect(reg_check(B, 512, "b"), true, "library entry survives the foreign one's removal");
  reg_take_error();
  const uint64_t t2 = reg_foreign(lib + 128, 4096);
  expect(reg_check(lib + 128, 2048, "c"), true, "foreign entry covers beyond the library's");
  reg_unforeign(t2);
  expect(reg_check(lib + 128, 2048, "d"), false, "after removal only the library's extent counts");
  std::string e_main = reg_take_error();
  expect(!e_main.empty(), true, "failure recorded for this thread");
  std::string e_other = "x";
  std::thread th([&] {
    reg_check(nullptr, 16, "other thread");
    e_other = reg_take_error();
  });
  th.join();
  expect(reg_take_error().empty(), true, "another thread's failure is not this thread's");
  expect(e_other.find("other thread") != std::string::npos, true, "the other thread reads its own failure");
  reg_free(B);
  expect(reg_check(B, 16, "e"), false, "freed");
  std::printf(fails ? "registry: %d failures\n" : "registry ok\n", fails);
  return fails ? 1 : 0;
}
