"""Build of the CUDA library libqmcrt.so (sm_103a) from csrc/.

Generates _build/gen/qmcrt_tables.h (Sobol direction numbers, Niederreiter generator
columns and Halton bases as table initialisers) and compiles each translation unit with nvcc in
parallel, then links one shared library.  The Sobol table is computed here from the
Joe & Kuo (2008) primitive polynomials and initial values that ship with SciPy, by
the Bratley-Fox recurrence m_k = 2 a_1 m_(k-1) ^ ... ^ 2^(s-1) a_(s-1) m_(k-s+1)
^ 2^s m_(k-s) ^ m_(k-s); the direction number of bit k is m_(k+1) 2^(31-k).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libqmcrt.so")
MAX_DIMS = 256
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["qmcrt_api.cu", "qmcrt_points.cu", "qmcrt_trace_single.cu", "qmcrt_trace_multiple.cu",
           "qmcrt_noalloc.cu", "qmcrt_batch.cu", "qmcrt_mlp.cu", "qmcrt_flow.cu", "qmcrt_warp_fused.cu",
           "qmcrt_trace_observers.cu", "qmcrt_direct.cu", "qmcrt_wavefront.cu", "qmcrt_host.cu",
           "qmcrt_sky.cu", "qmcrt_tail.cu"]


def _joe_kuo():
    import numpy as np
    import scipy

    d = np.load(os.path.join(os.path.dirname(scipy.__file__), "stats", "_sobol_direction_numbers.npz"))
    return d["poly"], d["vinit"]


def sobol_direction_table(dims: int = MAX_DIMS) -> list[list[int]]:
    poly, vinit = _joe_kuo()
    table = []
    for d in range(dims):
        if d == 0:
            m = [1] * 32
        else:
            p = int(poly[d])
            s = p.bit_length() - 1
            m = [int(vinit[d][j]) for j in range(s)]
            for k in range(s, 32):
                new = m[k - s] ^ (m[k - s] << s)
                for j in range(1, s):
                    if (p >> (s - j)) & 1:
                        new ^= m[k - j] << j
                m.append(new)
        table.append([(m[k] << (31 - k)) & 0xFFFFFFFF for k in range(32)])
    return table


def _gf2_deg(p: int) -> int:
    return p.bit_length() - 1


def _gf2_is_irreducible(p: int) -> bool:
    d = _gf2_deg(p)
    if d < 1:
        return False
    for q in range(2, 1 << (d // 2 + 1)):
        if _gf2_deg(q) > d // 2:
            break
        r = p
        while r and _gf2_deg(r) >= _gf2_deg(q):
            r ^= q << (_gf2_deg(r) - _gf2_deg(q))
        if r == 0:
            return False
    return True


def niederreiter_table(dims: int = MAX_DIMS) -> list[list[int]]:
    """Generator-matrix columns of the base-2 Niederreiter sequence (Niederreiter 1988):
    dimension j uses the j-th irreducible polynomial p over GF(2) (by degree, then
    value); for output digit r = q e + u (e = deg p) and input digit k the entry is the
    coefficient of t^(k-r) in the power series (t^e p(1/t))^-(q+1).  Column k holds
    output digit r at bit 31 - r."""
    table, p = [], 1
    for _ in range(dims):
        p += 1
        while not _gf2_is_irreducible(p):
            p += 1
        e = _gf2_deg(p)
        rev = [(p >> (e - i)) & 1 for i in range(e + 1)]  # coefficients of t^e p(1/t)
        inv = []
        for n in range(32):  # 1 / rev(t) by long division over GF(2)
            c = 1 if n == 0 else 0
            for i in range(1, min(n, e) + 1):
                c ^= rev[i] & inv[n - i]
            inv.append(c)

        def mul(a, b):
            return [sum(a[i] & b[n - i] for i in range(n + 1)) & 1 for n in range(32)]

        powers = [inv]  # powers[q] = rev^-(q+1)
        cols = [0] * 32
        for r in range(32):
            q = r // e
            while len(powers) <= q:
                powers.append(mul(powers[-1], inv))
            for k in range(r, 32):
                if powers[q][k - r]:
                    cols[k] |= 1 << (31 - r)
        table.append(cols)
    return table


def primes(n: int = MAX_DIMS) -> list[int]:
    out, c = [], 2
    while len(out) < n:
        if all(c % q for q in out if q * q <= c):
            out.append(c)
        c += 1
    return out


SOBOL_BYTE_DIMS = 8


def sobol_byte_table(V: list[list[int]], dims: int = SOBOL_BYTE_DIMS) -> list[list[list[int]]]:
    """T[d][b][v]: XOR of the direction numbers V[d][8 b + k] over the set bits k of the
    byte v, so that a coordinate is the XOR of four lookups, one per byte of the Gray code."""
    out = []
    for d in range(dims):
        per = []
        for b in range(4):
            row = [0] * 256
            for v in range(1, 256):
                low = v & -v
                row[v] = row[v ^ low] ^ V[d][8 * b + low.bit_length() - 1]
            per.append(row)
        out.append(per)
    return out


def write_tables() -> str:
    os.makedirs(GEN, exist_ok=True)
    path = os.path.join(GEN, "qmcrt_tables.h")
    V = sobol_direction_table()
    lines = ["/* generated by build.py: Sobol direction numbers (Joe-Kuo), Niederreiter columns, Halton bases */",
             "#pragma once",
             f"#define QMCRT_GEN_DIMS {MAX_DIMS}",
             "#define QMCRT_GEN_SOBOL_V_INIT { \\"]
    for row in V:
        lines.append("  {" + ",".join(f"0x{v:08x}u" for v in row) + "}, \\")
    lines.append("}")
    lines.append(f"#define QMCRT_GEN_SOBOL_BYTE_DIMS {SOBOL_BYTE_DIMS}")
    lines.append("#define QMCRT_GEN_SOBOL_BYTE_INIT { \\")
    for per in sobol_byte_table(V, SOBOL_BYTE_DIMS):
        lines.append("  { \\")
        for row in per:
            lines.append("    {" + ",".join(f"0x{v:08x}u" for v in row) + "}, \\")
        lines.append("  }, \\")
    lines.append("}")
    lines.append("#define QMCRT_GEN_PRIMES_INIT {" + ",".join(f"{p}u" for p in primes()) + "}")
    lines.append("#define QMCRT_GEN_NIED_V_INIT { \\")
    for row in niederreiter_table():
        lines.append("  {" + ",".join(f"0x{v:08x}u" for v in row) + "}, \\")
    lines.append("}")
    text = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    write_tables()
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "qmcrt.h"),
                                                                 os.path.join(GEN, "qmcrt_tables.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", GEN, "-I", CSRC] + (extra_flags or [])
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [_nvcc()] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode())
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
