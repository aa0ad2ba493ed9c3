"""Builds the CUDA library ``libmdilr.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled by nvcc in parallel, then linked
into one shared library (CUDA runtime linked statically) next to this file.
Rebuilds only what changed.  Run ``python -m paper_2404_08867_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import struct
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
GEN = os.path.join(OBJ, "gen")
LIB = os.path.join(PKG, "libmdilr.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "-I", INCLUDE, "-I", CSRC, "-I", GEN, "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmdilr.so")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + glob.glob(os.path.join(GEN, "*.inc"))


def _f32(v: float) -> float:
    return struct.unpack("<f", struct.pack("<f", v))[0]


def exp2_table_source() -> str:
    """2^(j/256), j = 0..255, as float pairs (hi = v rounded to float, lo = v - hi
    rounded to float; v - hi is exact in double), written as hex literals: the table
    of the double-float exp, so that no kernel computes it in FP64 at run time."""
    rows = []
    for j in range(256):
        v = 2.0 ** (j / 256.0)
        hi = _f32(v)
        lo = _f32(v - hi)
        rows.append(f"    {{{hi.hex()}f, {lo.hex()}f}},")
    return ("// Generated by build.py: 2^(j/256) for j = 0..255 as float pairs (hi, lo).\n"
            "static __device__ const float2 kExp2TableGen[256] = {\n" + "\n".join(rows) + "\n};\n")


def exp64_constants_source() -> str:
    """Constants of the FP64 table-driven exp (Tang's method) from their
    definitions, evaluated with 60-digit decimal arithmetic and rounded once to
    double: 2^(j/256) for j = 0..255; 256/ln2 (only used to pick the table index);
    ln2/256 split as L1 + L2 with L1 holding 33 significant bits, so that n L1 is
    exact for |n| < 2^20."""
    import decimal
    from fractions import Fraction
    ctx = decimal.Context(prec=60)
    ln2 = ctx.ln(decimal.Decimal(2))
    L = Fraction(ln2) / 256
    e = 0
    while Fraction(2) ** e <= L:
        e += 1
    while Fraction(2) ** e > L:
        e -= 1
    scale = Fraction(2) ** (32 - e)
    L1 = Fraction(round(L * scale)) / scale
    L2 = float(L - L1)
    inv = float(Fraction(256) / Fraction(ln2))
    rows = []
    for j in range(256):
        v = ctx.power(decimal.Decimal(2), ctx.divide(decimal.Decimal(j), decimal.Decimal(256)))
        rows.append(f"    {float(v).hex()},")
    return ("// Generated by build.py: constants of the FP64 table-driven exp.\n"
            f"static constexpr double kExp64Inv = {inv.hex()};  // 256 / ln2\n"
            f"static constexpr double kExp64L1 = {float(L1).hex()};  // ln2/256, 33 significant bits\n"
            f"static constexpr double kExp64L2 = {L2.hex()};  // ln2/256 - L1\n"
            "static __device__ const double kExp2TableD[256] = {\n" + "\n".join(rows) + "\n};\n")


def _dec_pi(ctx):
    """pi by Machin's formula, 16 atan(1/5) - 4 atan(1/239), in the context's precision."""
    import decimal

    def atan_inv(x):
        x = decimal.Decimal(x)
        term = ctx.divide(decimal.Decimal(1), x)
        x2 = x * x
        total, k, sign = term, 1, -1
        while True:
            term = ctx.divide(term, x2)
            t = ctx.divide(term, decimal.Decimal(2 * k + 1))
            if t == 0:
                return total
            total = ctx.add(total, t if sign > 0 else -t)
            k, sign = k + 1, -sign

    return ctx.subtract(ctx.multiply(16, atan_inv(5)), ctx.multiply(4, atan_inv(239)))


def _dec_cos_sin(theta, ctx):
    """cos and sin of theta (|theta| <= pi) by their Taylor series in the context's
    precision (the terms fall below 10^-60 well before the 80th)."""
    import decimal
    c = s = decimal.Decimal(0)
    term = decimal.Decimal(1)  # theta^k / k!
    for k in range(0, 160):
        if k % 4 == 0:
            c = ctx.add(c, term)
        elif k % 4 == 1:
            s = ctx.add(s, term)
        elif k % 4 == 2:
            c = ctx.subtract(c, term)
        else:
            s = ctx.subtract(s, term)
        term = ctx.divide(ctx.multiply(term, theta), decimal.Decimal(k + 1))
    return c, s


def cheb_table_source(pmax: int = 32) -> str:
    """Chebyshev points of the first kind on [0, 1] and their barycentric weights,
    xi_p = (1 + cos(theta_p)) / 2 and bw_p = (-1)^p sin(theta_p), theta_p =
    pi (2p + 1) / (2P), for every P = 1..pmax, from these definitions in 60-digit
    decimal arithmetic, each rounded once to double; the entries of P start at
    P (P - 1) / 2.  No kernel evaluates them in FP64 at run time."""
    import decimal
    ctx = decimal.Context(prec=70)
    pi = _dec_pi(ctx)
    xs, ws = [], []
    for P in range(1, pmax + 1):
        for p in range(P):
            theta = ctx.divide(ctx.multiply(pi, decimal.Decimal(2 * p + 1)), decimal.Decimal(2 * P))
            c, s = _dec_cos_sin(theta, ctx)
            xs.append(float(ctx.divide(ctx.add(decimal.Decimal(1), c), decimal.Decimal(2))))
            ws.append(float(s if p % 2 == 0 else -s))
    n = len(xs)
    body_x = "\n".join(f"    {v.hex()}," for v in xs)
    body_w = "\n".join(f"    {v.hex()}," for v in ws)
    return ("// Generated by build.py: Chebyshev points of the first kind on [0, 1] and their\n"
            f"// barycentric weights for P = 1..{pmax}; the entries of P start at P (P - 1) / 2.\n"
            f"static constexpr int kChebTablePMax = {pmax};\n"
            f"static __device__ const double kChebXiGen[{n}] = {{\n{body_x}\n}};\n"
            f"static __device__ const double kChebBwGen[{n}] = {{\n{body_w}\n}};\n")


def _write_generated():
    os.makedirs(GEN, exist_ok=True)
    _write_if_changed(os.path.join(GEN, "mdi_exp64_consts.inc"), exp64_constants_source())
    _write_if_changed(os.path.join(GEN, "mdi_cheb_table.inc"), cheb_table_source())
    path = os.path.join(GEN, "mdi_exp2_table.inc")
    src = exp2_table_source()
    if not os.path.exists(path) or open(path).read() != src:
        with open(path + ".tmp", "w") as f:
            f.write(src)
        os.replace(path + ".tmp", path)


def _write_if_changed(path: str, src: str):
    if not os.path.exists(path) or open(path).read() != src:
        with open(path + ".tmp", "w") as f:
            f.write(src)
        os.replace(path + ".tmp", path)


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra) -> str:
    obj = os.path.join(OBJ, os.path.basename(src) + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [_nvcc()] + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OBJ, exist_ok=True)
    _write_generated()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra_flags), sources))
    if _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    flags = sys.argv[1:]
    build(verbose=True, extra_flags=flags)
