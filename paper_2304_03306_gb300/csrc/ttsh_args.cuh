// ttsh_args.cuh - kernel argument block of a domain, built from its precision-erased
// description (shared by the per-launch kernels and the persistent batched stepper, so both
// compute with the same constants).
#pragma once

#include <cmath>

#include "ttsh_kernels.cuh"
#include "ttsh_ops.h"

namespace ttsh {

template <typename T>
inline Args<T> make_args(const DomainDev& d) {
  Args<T> a;
  a.what = static_cast<cplx<T>*>(d.what);
  a.vmean = static_cast<T*>(d.vmean);
  a.K = static_cast<T*>(d.K);
  a.G = static_cast<cplx<T>*>(d.G);
  a.Rr = static_cast<cplx<T>*>(d.Rr);
  a.tw = static_cast<const cplx<T>*>(d.tw);
  a.real = d.real;
  a.part = d.part;
  a.rec = d.rec;
  a.recctl = static_cast<RecCtl*>(d.recctl);
  a.err = d.err;
  a.aux = d.out ? d.out + 5 : nullptr;
  a.tma = 0;
  const double dk = 2.0 * 3.14159265358979323846264338327950288 / ((double)d.n * d.dx);
  a.a = (T)d.a;
  a.b = (T)d.b;
  a.lam = (T)d.lam;
  a.gv = (T)d.gv;
  a.gw = (T)d.gw;
  a.dt = (T)d.dt;
  a.dk = (T)dk;
  a.mean_decay = (T)exp((d.a - 1.0) * d.dt);
  a.dx = d.dx;
  a.cx = d.cx;
  a.cy = d.cy;
  return a;
}

}  // namespace ttsh
