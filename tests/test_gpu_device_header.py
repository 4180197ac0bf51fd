"""The device header used from a user's own kernel (the paper's Listing 1
shape): constructor + next() inside the kernel, state stored back."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    assert nvcc, "nvcc is needed to build the user kernel"
    out = str(tmp_path_factory.mktemp("user") / "liblisting1.so")
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "cuda", "listing1_user_kernel.cu"),
                    "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.run_listing1.restype = ctypes.c_int
    lib.run_listing1.argtypes = [ctypes.POINTER(srng.DevView), ctypes.c_void_p, ctypes.c_int]
    lib.run_user_threefry.restype = ctypes.c_int
    lib.run_user_threefry.argtypes = [ctypes.POINTER(srng.DevView), ctypes.c_void_p, ctypes.c_int]
    lib.run_user_threefry64.restype = ctypes.c_int
    lib.run_user_threefry64.argtypes = [ctypes.POINTER(srng.DevView), ctypes.c_void_p, ctypes.c_int]
    lib.run_user_next4.restype = ctypes.c_int
    lib.run_user_next4.argtypes = [ctypes.POINTER(srng.DevView), ctypes.c_void_p, ctypes.c_int]
    lib.run_user_offset.restype = ctypes.c_int
    lib.run_user_offset.argtypes = [ctypes.POINTER(srng.DevView), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.run_user_normals.restype = ctypes.c_int
    lib.run_user_normals.argtypes = [ctypes.POINTER(srng.DevView), ctypes.c_void_p, ctypes.c_int]
    return lib


def test_mrg_listing1_kernel(user_lib):
    n_streams, per = 1000, 7
    h = srng.srng_create_from_state([12345] * 6, n_streams, srng.SRNG_SPACING_STREAM)
    try:
        v = srng.srng_get_device_view(h)
        out = torch.empty(n_streams * per, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        assert user_lib.run_listing1(ctypes.byref(v), out.data_ptr(), per) == 0
        ref, _ = O.mrg_bulk(O.mrg_stream_starts([12345] * 6, 127, 0, n_streams), 2 * per, O.OUT_F32)
        got = out.cpu().numpy().reshape(n_streams, per)
        assert np.array_equal(got.view(np.uint32), ref[:, :per].view(np.uint32))
        # the state was stored back: the library's generate continues the streams
        nxt = torch.empty(n_streams * per, dtype=torch.float32, device="cuda")
        srng.srng_generate(h, 0, n_streams, per, srng.SRNG_OUT_F32, nxt)
        torch.cuda.synchronize()
        assert np.array_equal(nxt.cpu().numpy().reshape(n_streams, per).view(np.uint32), ref[:, per:].view(np.uint32))
    finally:
        srng.srng_destroy(h)


def test_philox_listing1_kernel(user_lib):
    n_streams, per = 300, 9
    seed = 0xC0FFEE
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, seed, n_streams)
    try:
        srng.srng_jump(h, 0, n_streams, srng.SRNG_JUMP_DRAWS, 3)  # start mid-block
        v = srng.srng_get_device_view(h)
        out = torch.empty(n_streams * per, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        assert user_lib.run_listing1(ctypes.byref(v), out.data_ptr(), per) == 0
        ref, _ = O.philox_bulk((seed, 0), 0, [3] * n_streams, per, O.OUT_U32)
        assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(n_streams, per), ref)
        pos = np.zeros(n_streams, dtype=np.uint64)
        srng.srng_get_state(h, 0, n_streams, pos)
        assert np.all(pos == 3 + per)
    finally:
        srng.srng_destroy(h)


@pytest.mark.parametrize("gen,start", [(srng.SRNG_THREEFRY4X32_20, 3), (srng.SRNG_THREEFRY4X64_20, 3),
                                       (srng.SRNG_THREEFRY4X64_20, 6)])
def test_user_kernel_threefry(user_lib, gen, start):
    """srng::Threefry4x32_20 / Threefry4x64_20 in a user kernel: draws equal
    the oracle's and the stored positions let the library continue the
    streams."""
    n_streams, per, seed = 300, 9, 0xC0FFEE
    h = srng.srng_create(gen, seed, n_streams)
    try:
        srng.srng_jump(h, 0, n_streams, srng.SRNG_JUMP_DRAWS, start)
        v = srng.srng_get_device_view(h)
        out = torch.empty(n_streams * per, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        if gen == srng.SRNG_THREEFRY4X32_20:
            assert user_lib.run_user_threefry(ctypes.byref(v), out.data_ptr(), per) == 0
            ref, _ = O.threefry_bulk(seed, 0, [start] * n_streams, 2 * per)
        else:
            assert user_lib.run_user_threefry64(ctypes.byref(v), out.data_ptr(), per) == 0
            ref, _ = O.threefry64_bulk(seed, 0, [start] * n_streams, 2 * per)
        assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(n_streams, per), ref[:, :per])
        nxt = torch.empty(n_streams * per, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, n_streams, per, srng.SRNG_OUT_U32, nxt)
        torch.cuda.synchronize()
        assert np.array_equal(nxt.cpu().numpy().view(np.uint32).reshape(n_streams, per), ref[:, per:])
    finally:
        srng.srng_destroy(h)


def _next4_reference(gen, seed, n_streams, start, n):
    """Oracle draws [start, start + n) of streams 0..n_streams-1 of a set made by srng_create(gen, seed)."""
    if gen == srng.SRNG_MRG32K3A:
        st = O.mrg_stream_starts(O.seed_expand(seed), 127, 0, n_streams)
        return O.mrg_bulk(st, start + n)[0][:, start:]
    if gen == srng.SRNG_TINYMT32:
        prm = O.tinymt32_find_params(seed, (n_streams + 255) // 256)
        st = O.tinymt32_stream_starts(seed & 0xFFFFFFFF, prm, 256, n_streams)
        return O.tinymt32_bulk(st, prm, 256, start + n)[0][:, start:]
    if gen == srng.SRNG_PHILOX4X32_10:
        return O.philox_bulk((seed & 0xFFFFFFFF, seed >> 32), 0, [start] * n_streams, n)[0]
    if gen == srng.SRNG_THREEFRY4X32_20:
        return O.threefry_bulk(seed, 0, [start] * n_streams, n)[0]
    return O.threefry64_bulk(seed, 0, [start] * n_streams, n)[0]


@pytest.mark.parametrize("gen", [srng.SRNG_MRG32K3A, srng.SRNG_PHILOX4X32_10, srng.SRNG_THREEFRY4X32_20,
                                 srng.SRNG_THREEFRY4X64_20, srng.SRNG_TINYMT32])
def test_user_kernel_next4(user_lib, gen):
    """next4() of every device class: four draws per call from any start
    (counter-based streams start 5 draws in, so the vectors straddle blocks),
    the state stored back so the library continues the streams."""
    n_streams, quads, seed = 300, 5, 0xC0FFEE
    start = 0 if gen in (srng.SRNG_MRG32K3A, srng.SRNG_TINYMT32) else 5
    h = srng.srng_create(gen, seed, n_streams)
    try:
        if start:
            srng.srng_jump(h, 0, n_streams, srng.SRNG_JUMP_DRAWS, start)
        v = srng.srng_get_device_view(h)
        out = torch.empty(n_streams * quads * 4, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        assert user_lib.run_user_next4(ctypes.byref(v), out.data_ptr(), quads) == 0
        ref = _next4_reference(gen, seed, n_streams, start, 4 * quads + 7)
        got = out.cpu().numpy().view(np.uint32).reshape(n_streams, 4 * quads)
        assert np.array_equal(got, ref[:, :4 * quads])
        nxt = torch.empty(n_streams * 7, dtype=torch.int32, device="cuda")
        srng.srng_generate(h, 0, n_streams, 7, srng.SRNG_OUT_U32, nxt)
        torch.cuda.synchronize()
        assert np.array_equal(nxt.cpu().numpy().view(np.uint32).reshape(n_streams, 7), ref[:, 4 * quads:])
    finally:
        srng.srng_destroy(h)


@pytest.mark.parametrize("gen", [srng.SRNG_MRG32K3A, srng.SRNG_PHILOX4X32_10, srng.SRNG_THREEFRY4X32_20,
                                 srng.SRNG_THREEFRY4X64_20])
def test_user_kernel_at_offset(user_lib, gen):
    """Stream handles built `offset` draws ahead inside the kernel: MRG32k3a by
    jump-ahead on the device (square and multiply, offsets up to 2^63 + 5),
    the counter-based ones by position; draws equal the oracle's."""
    n_streams, per, seed = 200, 9, 0xC0FFEE
    rng = np.random.default_rng(4)
    offs = rng.integers(0, 1 << 40, n_streams, dtype=np.uint64)
    offs[:6] = [0, 1, 2, 3, 7, 4096]
    offs[6:9] = [(1 << 63) + 5, (1 << 62) + 1, (1 << 40) + 3]
    h = srng.srng_create(gen, seed, n_streams)
    try:
        v = srng.srng_get_device_view(h)
        d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
        out = torch.empty(n_streams * per, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        assert user_lib.run_user_offset(ctypes.byref(v), out.data_ptr(), d_offs.data_ptr(), per) == 0
        got = out.cpu().numpy().view(np.uint32).reshape(n_streams, per)
        if gen == srng.SRNG_MRG32K3A:
            starts = O.mrg_stream_starts(O.seed_expand(seed), 127, 0, n_streams)
            want = np.stack([O.mrg_generate(O.mrg_jump(starts[i], int(offs[i])), per)[0] for i in range(n_streams)])
        elif gen == srng.SRNG_PHILOX4X32_10:
            want = np.stack([O.philox_generate((seed, 0), i, int(offs[i]), per) for i in range(n_streams)])
        elif gen == srng.SRNG_THREEFRY4X32_20:
            want = np.stack([O.threefry_generate(seed, i, int(offs[i]), per) for i in range(n_streams)])
        else:
            want = np.stack([O.threefry64_generate(seed, i, int(offs[i]), per) for i in range(n_streams)])
        assert np.array_equal(got, want)
    finally:
        srng.srng_destroy(h)


def test_user_kernel_normals(user_lib):
    """srng::dist::normal_pair inside a user kernel equals the oracle's
    Box-Muller on the oracle's Philox FP32 uniforms, bit for bit."""
    n_streams, pairs, seed = 257, 33, 0xC0FFEE
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, seed, n_streams)
    try:
        v = srng.srng_get_device_view(h)
        out = torch.empty(n_streams * 2 * pairs, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        assert user_lib.run_user_normals(ctypes.byref(v), out.data_ptr(), pairs) == 0
        u, _ = O.philox_bulk((seed, 0), 0, [0] * n_streams, 2 * pairs, O.OUT_F32)
        ref = O.transform(O.DIST_NORMAL, u.ravel())
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    finally:
        srng.srng_destroy(h)


@pytest.fixture(scope="module")
def paper_form_lib(tmp_path_factory):
    from paper_1412_8266_gb300 import _build
    nvcc = _build.nvcc()
    out = str(tmp_path_factory.mktemp("paper") / "libpaperform.so")
    pkg = os.path.dirname(srng.lib_path())
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-std=c++20",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "cuda", "listing1_paper_form.cu"), "-o", out,
                    "-L", pkg, "-lsrng", "-Xlinker", "-rpath=" + pkg], check=True)
    lib = ctypes.CDLL(out)
    lib.run_listing1_form.restype = ctypes.c_int
    lib.run_listing1_form.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    lib.run_philox_form.restype = ctypes.c_int
    lib.run_philox_form.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    lib.run_threefry64_form.restype = ctypes.c_int
    lib.run_threefry64_form.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    lib.run_tinymt_form.restype = ctypes.c_int
    lib.run_tinymt_form.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    lib.run_threefry_form.restype = ctypes.c_int
    lib.run_threefry_form.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    return lib


def test_paper_listing1_form(paper_form_lib):
    """RNG<float, Mrg32k3a> built without arguments, one draw per thread,
    launched three times: launch l holds draw l of every thread's stream."""
    block_num, thread_num, launches, seed = 37, 128, 3, 0x5EED
    n = block_num * thread_num
    out = torch.empty(launches * n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert paper_form_lib.run_listing1_form(out.data_ptr(), block_num, thread_num, launches, seed) == 0
    ref, _ = O.mrg_bulk(O.mrg_stream_starts(O.seed_expand(seed), 127, 0, n), launches, O.OUT_F32)
    got = out.cpu().numpy().reshape(launches, n).T
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_paper_form_philox(paper_form_lib):
    block_num, thread_num, seed = 5, 96, 0xC0FFEE
    n = block_num * thread_num
    out = torch.empty(2 * n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert paper_form_lib.run_philox_form(out.data_ptr(), block_num, thread_num, seed) == 0
    ref, _ = O.philox_bulk((seed, 0), 0, [0] * n, 2, O.OUT_U32)
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(n, 2), ref)


def test_paper_form_threefry(paper_form_lib):
    block_num, thread_num, seed = 7, 64, 0xBEEF
    n = block_num * thread_num
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert paper_form_lib.run_threefry_form(out.data_ptr(), block_num, thread_num, seed) == 0
    ref, _ = O.threefry_bulk(seed, 0, [0] * n, 1, O.OUT_F64)
    assert np.array_equal(out.cpu().numpy(), ref.ravel())


def test_paper_form_threefry64(paper_form_lib):
    block_num, thread_num, seed = 7, 64, 0xBEEF
    n = block_num * thread_num
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert paper_form_lib.run_threefry64_form(out.data_ptr(), block_num, thread_num, seed) == 0
    ref, _ = O.threefry64_bulk(seed, 0, [0] * n, 1, O.OUT_F64)
    assert np.array_equal(out.cpu().numpy(), ref.ravel())


def test_paper_form_tinymt(paper_form_lib):
    """RNG<float, TinyMT32> with 256-thread blocks: block b's threads share
    parameter set b (the paper's Sec. 4.2 hybrid) and thread t of the block
    takes substream t."""
    block_num, thread_num, seed = 3, 256, 0xFEED
    n = block_num * thread_num
    out = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert paper_form_lib.run_tinymt_form(out.data_ptr(), block_num, thread_num, seed) == 0
    prm = O.tinymt32_find_params(seed, block_num)
    st = O.tinymt32_stream_starts(seed & 0xFFFFFFFF, prm, 256, n)
    ref, _ = O.tinymt32_bulk(st, prm, 256, 2, O.OUT_F32)
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(n, 2), ref.view(np.uint32))


def test_mrg_f64_forms_agree_exhaustively(tmp_path):
    """The three forms of the MRG32k3a double the generation kernels mix -- built
    from integers, the FP64 multiply, and the one-FMA form -- agree bit for bit
    for every z in [1, m1] (the integer-built form is compared with the IEEE
    product in the conversion tests)."""
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    assert nvcc, "nvcc is needed to build the check"
    out = str(tmp_path / "libforms.so")
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "cuda", "mrg_f64_forms.cu"),
                    "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.run_mrg_f64_forms.restype = ctypes.c_int
    lib.run_mrg_f64_forms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_ulonglong),
                                      ctypes.POINTER(ctypes.c_ulonglong)]
    bad, first = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    assert lib.run_mrg_f64_forms(1, O.M1, ctypes.byref(bad), ctypes.byref(first)) == 0
    assert bad.value == 0, f"{bad.value} values differ, the first at z = {first.value}"
