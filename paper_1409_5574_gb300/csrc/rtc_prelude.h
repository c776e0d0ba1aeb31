// What the step kernels need from the C/C++ libraries when they are compiled
// at run time by NVRTC (which has no host headers): the fixed-width integer
// types and three type traits.  Included only under __CUDACC_RTC__.
#pragma once

typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;

namespace std {
template <class T, T v>
struct integral_constant {
  static constexpr T value = v;
  using value_type = T;
  using type = integral_constant;
  constexpr operator T() const { return v; }
};
template <class A, class B>
struct is_same : integral_constant<bool, false> {};
template <class A>
struct is_same<A, A> : integral_constant<bool, true> {};
template <bool B, class T, class F>
struct conditional {
  using type = T;
};
template <class T, class F>
struct conditional<false, T, F> {
  using type = F;
};
}  // namespace std
