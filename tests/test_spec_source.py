"""The kernel source that run-time specialisation compiles with NVRTC
(push_emit.cu and the headers it includes) compiles under NVRTC with the
specialised constants, for the table sampler's three launch forms, the
learned samplers and the Yee grid's plain and tile-staged kernels, without a
GPU.  The
library embeds the same files at build time; this keeps them free of host
code outside the __CUDACC_RTC__ guards."""
import ctypes
import os

import pytest

from paper_1409_5574_gb300 import build


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    try:
        return ctypes.CDLL(os.path.join(home, "lib64", "libnvrtc.so.13"))
    except OSError:
        pytest.skip("NVRTC not available")


# constants of a 0.8 um, a0 = 500 wave with 100 steps per period (exact
# float literals) and Philox round keys of an arbitrary key
DEFINES = [
    "-DPRAD_SPEC", "-DPRAD_SPEC_HALF_Q_DTN=(-0x1.015bfap-6f)", "-DPRAD_SPEC_DTN=(0x1.015bfap-5f)",
    "-DPRAD_SPEC_INV_DTN=(0x1.fd4bbap+4f)", "-DPRAD_SPEC_CN_DT=(0x1.09113p-14f)",
    "-DPRAD_SPEC_EPS_R15=(0x1.314cecp-18f)", "-DPRAD_SPEC_LL_COEF=(0x1.fda8d4p-32f)",
    "-DPRAD_SPEC_E0=(0x1.f4p+8f)", "-DPRAD_SPEC_KC=(0x1.45f306p-3f)",
    "-DPRAD_SPEC_KC_LO=(0x1.b9391p-28f)", "-DPRAD_SPEC_CP_DT=(0x1.2a3b4cp-12f)", "-DPRAD_SPEC_PHASE_STEP=92233720368547745ull",
    "-DPRAD_SPEC_ENSEMBLE=3u",
    "-DPRAD_SPEC_RKEY={" + ",".join("%du" % (1000003 * k + 7) for k in range(20)) + "}",
]


YEE = ["-DPRAD_SPEC_YEE", "-DPRAD_SPEC_NX=4096", "-DPRAD_SPEC_NY=4096", "-DPRAD_SPEC_NTX=128",
       "-DPRAD_SPEC_INV_DX=(0x1.45f306p+2f)", "-DPRAD_SPEC_INV_DY=(0x1.45f306p+2f)",
       "-DPRAD_SPEC_INV_DX_LO=(0x1.b9391p-23f)", "-DPRAD_SPEC_INV_DY_LO=(0x1.b9391p-23f)",
       "-DPRAD_SPEC_X0=(0x0p+0f)", "-DPRAD_SPEC_Y0=(0x0p+0f)",
       "-DPRAD_SPEC_LX=(0x1.921fb6p+9f)", "-DPRAD_SPEC_LY=(0x1.921fb6p+9f)"]

CASES = [(b"prad::k_push_emit<float, 1, %d, %d, false, true, %d>" % c, []) for c in
         [(0, 0, 4), (0, 1, 1), (0, 2, 3), (1, 0, 2), (2, 0, 4)]]
CASES += [(b"prad::k_push_emit<float, 2, 0, %d, false, true, 0>" % pf, YEE) for pf in (0, 2)]
CASES += [(b"prad::k_push_emit_tiled<float, false, true>", YEE)]


@pytest.mark.parametrize("expr,extra", CASES, ids=[c[0].decode().split("<")[0][6:] + "_"
                                                    + str(i) for i, c in enumerate(CASES)])
def test_kernel_source_compiles_under_nvrtc(expr, extra):
    nv = _nvrtc()
    paths = build.SPEC_SOURCES
    texts = [open(p, "rb").read() for p in paths]
    names = [os.path.basename(p).encode() for p in paths]
    nh = len(paths) - 1
    hdr = (ctypes.c_char_p * nh)(*texts[1:])
    inc = (ctypes.c_char_p * nh)(*names[1:])
    prog = ctypes.c_void_p()
    assert nv.nvrtcCreateProgram(ctypes.byref(prog), texts[0], names[0], nh, hdr, inc) == 0
    assert nv.nvrtcAddNameExpression(prog, expr) == 0
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    opts = [b"-arch=sm_103a", b"-std=c++17", b"-default-device",
            ("-I" + os.path.join(home, "include")).encode()] + [d.encode() for d in DEFINES + extra]
    argv = (ctypes.c_char_p * len(opts))(*opts)
    rc = nv.nvrtcCompileProgram(prog, len(opts), argv)
    n = ctypes.c_size_t()
    nv.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value + 1)
    nv.nvrtcGetProgramLog(prog, log)
    assert rc == 0, log.value.decode(errors="replace")[:2000]
    nbin = ctypes.c_size_t()
    assert nv.nvrtcGetCUBINSize(prog, ctypes.byref(nbin)) == 0
    assert nbin.value > 1000
    lowered = ctypes.c_char_p()
    assert nv.nvrtcGetLoweredName(prog, expr, ctypes.byref(lowered)) == 0
    assert lowered.value.startswith(b"_ZN4prad")
    nv.nvrtcDestroyProgram(ctypes.byref(prog))
