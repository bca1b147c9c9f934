"""Build libdgx.so: nvcc for sm_103a, one translation unit per (dim, precision,
degree) so the kernel templates compile in parallel, linked into one shared
library next to this file.  Run ``python -m paper_2607_16044_b300.build``.
"""
import concurrent.futures
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libdgx.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(os.path.dirname(HERE), "include")]
DEGREES = (1, 2, 3, 4, 5)

UNIT = """// generated by build.py: instantiation of the (D={D}, S={S}, P={P}) launch table
#include "dispatch.h"
{VJP_INCLUDE}
{TC_INCLUDE}
#include "dgip.cuh"
namespace dgx {{
namespace {{
using Sc = {S};
using O = Ops<{D}, {P}, Sc>;
inline const Mesh<Sc>& m(const void* M) {{ return *(const Mesh<Sc>*)M; }}
struct R {{
  static cudaError_t trace(const void* M, int V, const void* U, void* TU, cudaStream_t st) {{
    return O::template trace<Sc>(m(M), V, (const Sc*)U, (Sc*)TU, nullptr, st);
  }}
  static cudaError_t tr64(const void* M, int V, const double* U, void* TU, void* sh, cudaStream_t st) {{
    return O::template trace<double>(m(M), V, U, (Sc*)TU, (Sc*)sh, st);
  }}
  static cudaError_t br1(const void* M, int V, bool c, const void* U, const Work& w, cudaStream_t st) {{
    return O::br1(m(M), V, c, (const Sc*)U, w, st);
  }}
  static cudaError_t face(const void* M, bool v, bool c, const Work& w, cudaStream_t st) {{
    return O::face(m(M), v, c, w, st);
  }}
  static cudaError_t elem(const void* M, int V, bool v, bool c, const void* U, const Work& w, void* out,
                          cudaStream_t st) {{
    Stage<Sc> none{{}};
    return O::template elem<0>(m(M), V, v, c, (const Sc*)U, w, (Sc*)out, none, st);
  }}
  static cudaError_t elem_stage(const void* M, int V, bool v, bool c, const void* U, const Work& w, const void* sa,
                                cudaStream_t st) {{
    return O::template elem<1>(m(M), V, v, c, (const Sc*)U, w, nullptr, *(const Stage<Sc>*)sa, st);
  }}
  static cudaError_t elem_pipe(const void* M, int V, bool v, bool c, const void* U, const Work& w, void* out,
                               const void* sa, int nsm, cudaStream_t st, bool* used) {{
    if (sa) return O::template elem_pipe<1>(m(M), V, v, c, (const Sc*)U, w, nullptr, *(const Stage<Sc>*)sa, nsm, st,
                                           *used);
    Stage<Sc> none{{}};
    return O::template elem_pipe<0>(m(M), V, v, c, (const Sc*)U, w, (Sc*)out, none, nsm, st, *used);
  }}
{TC_FN}
  static size_t smem(int kind, int V) {{ return O::smem(kind, V); }}
}};
}}  // namespace
const Table* table_d{D}_{T}_p{P}() {{
  static const Table t = {{&R::trace, &R::tr64, &R::br1, &R::face, &R::elem, &R::elem_stage, &R::elem_pipe,
                          {TC_PTR}, &R::smem, {VJP_PTR}, dgip_table<{D}, {P}, Sc>()}};
  return &t;
}}
}}  // namespace dgx
"""

# degrees above the LLF/BR1 range: the DG-IP launch table alone (the point
# operator of over-integration with 7 or 8 points per direction)
DGIP_DEGREES = (6, 7)

DGIP_UNIT = """// generated by build.py: the DG-IP launch table alone for (D={D}, S={S}, P={P})
#include "dispatch.h"
#include "dgip.cuh"
namespace dgx {{
const void* dgip_only_d{D}_{T}_p{P}() {{ return dgip_table<{D}, {P}, {S}>(); }}
}}  // namespace dgx
"""

TC_FN = """  static cudaError_t elem_tc(const void* M, int tc, bool v, bool c, const void* U, const Work& w, void* out,
                             const void* sa, cudaStream_t st) {{
    return TcOps<{D}, {P}>::elem(m(M), tc, v, c, (const float*)U, w, (float*)out, (const Stage<float>*)sa, st);
  }}"""

DISPATCH = """// generated by build.py: degree dispatch
#include "dispatch.h"
namespace dgx {{
{DECLS}
{FUNCS}
}}  // namespace dgx
"""


def _vjp_available():
    return os.path.exists(os.path.join(CSRC, "vjp.cuh"))


def _write_sources():
    os.makedirs(BUILD, exist_ok=True)
    units = []
    decls, funcs = [], []
    vjp = _vjp_available()
    for D in (2, 3):
        for S, T in (("double", "f64"), ("float", "f32")):
            cases = []
            for P in DEGREES:
                name = f"table_d{D}_{T}_p{P}"
                decls.append(f"const Table* {name}();")
                cases.append(f"    case {P}: return {name}();")
                vjp_inc = '#include "vjp.cuh"' if vjp else ""
                vjp_ptr = f"vjp_table<{D}, {P}, {S}>()" if vjp else "nullptr"
                f32 = S == "float"
                src = UNIT.format(D=D, S=S, P=P, T=T, VJP_INCLUDE=vjp_inc, VJP_PTR=vjp_ptr,
                                  TC_INCLUDE='#include "kernels_tc.cuh"' if f32 else "",
                                  TC_FN=TC_FN.format(D=D, P=P) if f32 else "",
                                  TC_PTR="&R::elem_tc" if f32 else "nullptr")
                path = os.path.join(BUILD, f"unit_d{D}_{T}_p{P}.cu")
                _write_if_changed(path, src)
                units.append(path)
            funcs.append(f"const Table* table_d{D}_{T}(int P) {{\n  switch (P) {{\n" + "\n".join(cases)
                         + "\n    default: return nullptr;\n  }\n}")
            only = []
            for P in DGIP_DEGREES:
                name = f"dgip_only_d{D}_{T}_p{P}"
                decls.append(f"const void* {name}();")
                only.append(f"    case {P}: return {name}();")
                path = os.path.join(BUILD, f"dgip_unit_d{D}_{T}_p{P}.cu")
                _write_if_changed(path, DGIP_UNIT.format(D=D, S=S, P=P, T=T))
                units.append(path)
            funcs.append(f"const void* dgip_only_d{D}_{T}(int P) {{\n  switch (P) {{\n" + "\n".join(only)
                         + "\n    default: return nullptr;\n  }\n}")
    path = os.path.join(BUILD, "dispatch_gen.cu")
    _write_if_changed(path, DISPATCH.format(DECLS="\n".join(decls), FUNCS="\n".join(funcs)))
    units.append(path)
    units.append(os.path.join(CSRC, "host.cu"))
    units.append(os.path.join(CSRC, "noalloc.cu"))
    units.append(os.path.join(CSRC, "probe.cu"))
    units.append(os.path.join(CSRC, "batchp.cu"))
    units.append(os.path.join(CSRC, "hdg.cu"))
    units.append(os.path.join(CSRC, "oi.cu"))
    return units


def _write_if_changed(path, text):
    if os.path.exists(path) and open(path).read() == text:
        return
    with open(path, "w") as f:
        f.write(text)


def _deps_hash():
    h = hashlib.sha256()
    for root in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for name in sorted(os.listdir(root)):
            if name.endswith((".cuh", ".h")):  # headers; each unit's own text is in its key
                h.update(name.encode())
                h.update(open(os.path.join(root, name), "rb").read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _compile(src, deps):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    stamp = obj + ".stamp"
    key = deps + open(src).read()
    key = hashlib.sha256(key.encode()).hexdigest()
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
        return obj
    cmd = [NVCC, *ARCH, *FLAGS, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as f:
        f.write(key)
    return obj


def build(verbose=True, jobs=None):
    units = _write_sources()
    deps = _deps_hash()
    jobs = jobs or max(1, os.cpu_count() or 1)
    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, deps), units))
    cmd = [NVCC, *ARCH, "-shared", "-o", LIB, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build()
    sys.exit(0)
