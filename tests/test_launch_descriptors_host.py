"""Launch descriptors of large plans, checked on the CPU.

The library's host sources (planner, C ABI) are linked with
tests/host_launch_stubs.cpp, a stand-in CUDA runtime whose kernel launchers
log their descriptors instead of launching.  A plan is created, bound to a
fake device address range and run for one step on the bench's seeded
subset of slices; every logged launch is then checked:

* operands inside the arena: the result block of every key, and the span of
  A's and B's address bits from their offsets;
* the alignment that the kernels' 16-byte accesses need: result pairs of the
  streaming kernel with two or more columns per thread, the keyed kernel's
  results and packed right operands, the tensor-core kernels' operand bases
  and TMA maps (16-byte base, strides and inner box);
* the key tables and scratch regions inside the device allocation, 4-byte
  (tables) or 256-byte (scratch) aligned;
* the keyed kernel's row count a multiple of its rows per item.

The 53-qubit plans with 300,000 (TF32 split) and 1,000,000 (FP32)
bitstrings are workloads whose first step met a misaligned-address fault on
the GPU.
"""
import ctypes
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_05665_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

_RUN = textwrap.dedent("""
    import sys, ctypes
    sys.path.insert(0, {root!r})
    from paper_2108_05665_gb300 import binding as B, inputs
    import bench
    B.load({lib!r})
    w = inputs.WORKLOADS[{name!r}]
    circ = w.circuit(); bits = bench.load_bitstrings(w)
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3 if {prec!r} == "tf32x3" else B.XEB_PREC_FP32
    if w.n_qubits > 40:
        o.mem_budget = 200 << 30
    plan = B.Plan(circ, bits, opts=o)
    st = B.xeb_plan_stats(plan.handle)
    nb = B.xeb_plan_device_bytes(plan.handle)
    base = 0x100000000000
    B._check(B.load().xeb_plan_bind(plan.handle, ctypes.c_void_p(base), ctypes.c_size_t(nb), ctypes.c_void_p(None)))
    if st["n_slices"] > 4:
        B.xeb_set_slice_subset(plan.handle, 4.0 / st["n_slices"], 12345)
    B.xeb_set_bitstrings(plan.handle, base, len(bits), 0)
    B.xeb_amplitudes(plan.handle, base + nb, 0)
    print("ARENA", st["arena_bytes"], "DEVICE", nb)
""")


@pytest.fixture(scope="module")
def emu_lib(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime_api.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("hostemu")
    objs = []
    srcs = [os.path.join(CSRC, f) for f in ("capi.cpp", "plan.cpp", "anneal.cpp")]
    srcs.append(os.path.join(ROOT, "tests", "host_launch_stubs.cpp"))
    for s in srcs:
        o = str(d / (os.path.basename(s) + ".o"))
        subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-pthread", "-I", os.path.join(ROOT, "include"),
                        "-I", CSRC, "-I", CUDA_INC, "-c", s, "-o", o], check=True)
        objs.append(o)
    lib = str(d / "libxeb_emu.so")
    subprocess.run(["g++", "-shared", "-Wl,--no-undefined", "-o", lib, *objs, "-pthread"], check=True)
    return lib


def _parse(line):
    parts = line.split()
    d = {"kind": parts[0]}
    for p in parts[1:]:
        if "=" not in p:
            continue
        k, v = p.split("=", 1)
        if v.endswith(","):
            d[k] = [int(x) for x in v.strip(",").split(",")]
        elif v == "":
            d[k] = []
        else:
            try:
                d[k] = int(v)
            except ValueError:
                d[k] = v
    return d


def _emulate(emu_lib, tmp_path, name, prec):
    log = str(tmp_path / ("%s_%s.log" % (name, prec)))
    env = dict(os.environ, XEB_EMU_LOG=log)
    code = _RUN.format(root=ROOT, lib=emu_lib, name=name, prec=prec)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    tail = [l for l in r.stdout.splitlines() if l.startswith("ARENA")][-1].split()
    arena, device = int(tail[1]) // 8, int(tail[3])
    return [_parse(l) for l in open(log)], arena, device


def _span(bits):
    return sum(1 << b for b in bits)


def _check_launches(launches, arena, device):
    problems = []
    gemms = 0   # contraction launches, SIMT and tensor-core
    for d in launches:
        k = d["kind"]
        if k in ("keyed", "stream", "memo", "memo_prep") or k.startswith("gemm"):
            gemms += 1
            M, N, kv = d["M"], d["N"], d["kv"]
            where = "%s M=%d N=%d K=%d kv=%d" % (k, M, N, d["K"], kv)
            for f in ("a_off", "b_off", "c_off", "a_key", "b_key", "c_key"):
                if d[f] < 0:
                    problems.append(where + ": negative " + f)
            c_end = d["c_off"] + (kv - 1) * d["c_key"] + M * N if kv > 1 else d["c_off"] + M * N
            if c_end > arena:
                problems.append(where + ": result beyond the arena")
            if d["a_off"] + _span(d["apm"] + d["apk"]) >= arena or d["b_off"] + _span(d["bpk"] + d["bpn"]) >= arena:
                problems.append(where + ": operand span beyond the arena")
            for t in ("uL", "uR", "gstart"):
                if d[t] >= 0 and (d[t] % 4 or d[t] >= device):
                    problems.append(where + ": key table " + t)
            if max(d["apm"] + d["apk"] + d["bpk"] + d["bpn"] + [0]) > 47:
                problems.append(where + ": address bit above 47")
            if k == "stream" and d["npt"] >= 2 and (d["c_off"] % 2 or (kv > 1 and d["c_key"] % 2) or N % 2
                                                   or not d["c_natural"]):
                problems.append(where + ": 16-byte result pairs misaligned")
            if k == "keyed":
                if d["c_off"] % 2 or d["c_key"] % 2:
                    problems.append(where + ": keyed results misaligned")
                if d["scratch"] % 256 or d["scratch"] >= device:
                    problems.append(where + ": keyed scratch")
                if M % (32 * d["rpt"]):
                    problems.append(where + ": rows not a multiple of the item")
                if max(d["apk"] + [0]) > 30:
                    problems.append(where + ": 32-bit summed-index offsets overflow")
            if k in ("memo", "memo_prep") and (d["scratch"] % 256 or d["scratch"] >= device):
                problems.append(where + ": memo scratch")
        elif k == "tc2":
            gemms += 1
            if d["a_off"] % 2 or d["c_off"] % 2 or d["b_off"] % 2:
                problems.append("tc2 M=%d: operand base not 16-byte aligned" % d["M"])
        elif k == "tckd":
            gemms += 1
            if d["c_off"] % 2:
                problems.append("tckd: result base odd")
        elif k == "tmap":
            rank = d["rank"]
            if d["addr"] % 16 or any(d["stride%d" % i] % 16 for i in range(rank - 1)) or (d["box0"] * 4) % 16:
                problems.append("tmap: base, stride or inner box not a multiple of 16 bytes")
            if d["addr"] >= device:
                problems.append("tmap: base beyond the allocation")
    return gemms, problems


@pytest.mark.parametrize("name,prec", [("grid5x6_m14_k10000", "tf32x3"), ("grid6x9m1_m12_k300000", "tf32x3"),
                                       ("grid6x9m1_m14_k1000000", "fp32")])
def test_launch_descriptors_are_in_range_and_aligned(emu_lib, tmp_path, name, prec):
    launches, arena, device = _emulate(emu_lib, tmp_path, name, prec)
    gemms, problems = _check_launches(launches, arena, device)
    assert gemms > 20
    assert not problems, problems[:10]
    if name.startswith("grid5x6"):
        # the unsliced 30-qubit plan runs its sweep on the TMA tensor-core form
        assert sum(1 for d in launches if d["kind"] == "tc2" and d["tma"]) >= 20
        assert sum(1 for d in launches if d["kind"] == "tmap") >= 20
        # and its large K = 1 outer product (2^24 x 64 results) meets the
        # outer-product kernel's conditions (natural layouts, even offsets)
        outer = [d for d in launches if d["kind"] == "stream" and _outer_fits(d)]
        assert any(d["M"] == 1 << 24 and d["N"] == 64 for d in outer)


def _outer_fits(d):
    """The conditions under which the streaming launcher runs k_outer."""
    M, N = d["M"], d["N"]
    return (d["K"] == 1 and d["kv"] == 1 and d["n_groups"] == 1 and d["c_natural"] and d["nak"] == 0
            and d["nbk"] == 0 and 2 <= N <= 512 and N & (N - 1) == 0 and M == 1 << d["nam"] and N == 1 << d["nbn"]
            and d["apm"] == list(range(d["nam"])) and d["bpn"] == list(range(d["nbn"]))
            and d["c_off"] % 2 == 0 and d["b_off"] % 2 == 0 and d["b_key"] % 2 == 0)


def test_stub_helpers_match_the_library(emu_lib):
    """The stand-in copies of the library's host-side size and eligibility
    helpers (defined in its CUDA sources) give the library's answers."""
    real = os.path.join(ROOT, "paper_2108_05665_gb300", "_lib", "libxeb.so")
    if not os.path.exists(real):
        pytest.skip("library not built")
    a, b = ctypes.CDLL(real), ctypes.CDLL(emu_lib)
    L3 = [ctypes.c_int64] * 3
    for sym, args, res in [("_ZN4xebk10keyed_fitsElll", L3, ctypes.c_bool),
                           ("_ZN4xebk16keyed_fits_rows2Elll", L3, ctypes.c_bool),
                           ("_ZN4xebk19keyed_scratch_bytesElll", L3, ctypes.c_size_t)]:
        fa, fb = a[sym], b[sym]
        for f in (fa, fb):
            f.argtypes, f.restype = args, res
        for M in (32, 48, 64, 1 << 20):
            for N in (1, 2, 3, 16, 32):
                for K in (2, 4, 16, 32, 64):
                    assert fa(M, N, K) == fb(M, N, K), (sym, M, N, K)
    fa, fb = a["_ZN4xebk18memo_scratch_bytesElllm"], b["_ZN4xebk18memo_scratch_bytesElllm"]
    for f in (fa, fb):
        f.argtypes, f.restype = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_size_t], ctypes.c_size_t
    for args in [(1, 16, 16, 8), (300, 3000, 16, 8), (7, 9, 4, 16)]:
        assert fa(*args) == fb(*args)
    fa, fb = a["_ZN4xebk23trie_sort_scratch_bytesEi"], b["_ZN4xebk23trie_sort_scratch_bytesEi"]
    for f in (fa, fb):
        f.argtypes, f.restype = [ctypes.c_int], ctypes.c_size_t
    for k in (1, 4095, 4096, 300000, 1000000):
        assert fa(k) == fb(k)
