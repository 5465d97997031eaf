"""GPU parity of the batched plan (fbf_plan_create / fbf_filter_batched): every
image of an uneven batch, each with its own window, range scale and order K,
against the FP64 oracle and against the single-image filter, for the
autotuned FP32 / AUTO plans, the per-image tensor-core plans and the
persistent tensor-core plan of the single FP16 form."""
import numpy as np
import pytest

import oracle as O
from paper_1603_08081_gb300.synth import make_batch_specs, make_image

pytestmark = pytest.mark.gpu

TOL_FP32 = 0.05  # same regression bound as the single-image FP32 form (0.5 gray contract)


@pytest.fixture(scope="module")
def fbf():
    import torch  # noqa: F401

    from paper_1603_08081_gb300 import build

    build.build()
    from paper_1603_08081_gb300 import fbf as mod

    return mod


def _run_plan(fbf, imgs, specs, border="reflect", form="fp32"):
    import torch

    xs = [torch.from_numpy(im).cuda() for im in imgs]
    ys = [torch.full(im.shape, float("nan"), dtype=torch.float32, device="cuda") for im in imgs]
    plan = fbf.fbf_plan_create(xs, ys, specs, form, border)
    for y in ys:  # autotuning wrote the outputs: clear them before the timed-free replay
        y.fill_(float("nan"))
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    return plan, xs, ys


@pytest.mark.parametrize("border", ["reflect", "truncate"])
def test_uneven_batch_matches_oracle(fbf, border):
    shapes = [(70, 90), (33, 200), (256, 40), (5, 7), (130, 131), (1, 64)]
    specs = [dict(sigma_s=3.0, sigma_r=30.0), dict(sigma_s=0.7, sigma_r=15.0), dict(sigma_s=6.0, sigma_r=50.0),
             dict(sigma_s=10.0, sigma_r=20.0), dict(sigma_s=2.0, sigma_r=60.0, eps=1e-2),
             dict(sigma_s=4.0, sigma_r=25.0, W=3, spatial="box")]
    imgs = [make_image(h, w, seed=1300 + k) for k, (h, w) in enumerate(shapes)]
    plan, xs, ys = _run_plan(fbf, imgs, specs, border)
    ni, nt = plan.size()
    assert ni == len(imgs) and nt > len(imgs)
    bd = O.BORDER_REFLECT if border == "reflect" else O.BORDER_TRUNCATE
    for im, sp, y in zip(imgs, specs, ys):
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, sp.get("eps", 1e-3))
        W = sp.get("W", int(np.ceil(3 * sp["sigma_s"] - 1e-12)))
        w1 = O.weights_1d(O.SPATIAL_BOX if sp.get("spatial") == "box" else O.SPATIAL_GAUSSIAN, sp["sigma_s"], W)
        ref = O.alg1(im, w1, bd, np.array(c.coefficients), 255.0)[0]
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_FP32
    plan.destroy()


def test_batch_equals_single_image_filter_and_relaunches(fbf):
    """A 64-image batch shaped like the uneven workload (smaller sizes): each
    output equals the single-image FP32 filter, and a second graph launch gives
    the same outputs (the work counter is reset inside the graph)."""
    import torch

    specs_raw = make_batch_specs(64, seed=1399, lo=48, hi=400)
    imgs = [make_image(h, w, seed=s) for (h, w, _, _, s) in specs_raw]
    specs = [dict(sigma_s=ss, sigma_r=sr) for (_, _, ss, sr, _) in specs_raw]
    plan, xs, ys = _run_plan(fbf, imgs, specs)
    first = [y.clone() for y in ys]
    for y in ys:
        y.fill_(float("nan"))
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    for y0, y1 in zip(first, ys):
        assert torch.equal(y0, y1)
    for x, y, sp in zip(xs, ys, specs):
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, 1e-3)
        p = fbf.make_params(c, sp["sigma_s"])
        single = fbf.fbf_filter(p, x)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(single - y)).item() <= 1e-4
    plan.destroy()


def test_empty_plan_and_invalid_arguments(fbf):
    import ctypes as C

    import torch

    plan = fbf.fbf_plan_create([], [], [])
    assert plan.size() == (0, 0)
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    plan.destroy()
    h = C.c_void_p()
    arr = (fbf.fbf_image_desc * 1)()  # sigma_r = 0: the fit rejects it
    assert fbf.lib.fbf_plan_create(arr, 1, fbf.FBF_FORM_TC_FP16, 0, C.byref(h)) == fbf.FBF_ERR_INVALID_ARGUMENT
    assert fbf.lib.fbf_plan_create(arr, 1, 9, 0, C.byref(h)) == fbf.FBF_ERR_INVALID_ARGUMENT


@pytest.mark.parametrize("form", ["fp32", "auto"])
def test_autotuned_plan_equals_its_schedule(fbf, form):
    """The autotuner keeps one of its candidates; whichever it keeps, every
    output equals the single-image filter of the matching form (per-image
    schedules replay exactly those kernels: bit-identical; the persistent
    kernels are the FP32 tile body with run-time taps: within 1e-4)."""
    import torch

    specs_raw = make_batch_specs(24, seed=1399, lo=64, hi=700)
    imgs = [make_image(h, w, seed=s) for (h, w, _, _, s) in specs_raw]
    specs = [dict(sigma_s=ss, sigma_r=sr) for (_, _, ss, sr, _) in specs_raw]
    specs[3] = dict(sigma_s=1.0, sigma_r=30.0, W=6, spatial="box")
    plan, xs, ys = _run_plan(fbf, imgs, specs, form=form)
    kind, ms = plan.schedule()
    assert kind in fbf.SCHEDULES and ms > 0
    per_form = {"per_image_fp32": "fp32", "per_image_form": form, "per_image_fp32_streams": "fp32",
                "per_image_form_streams": form}.get(kind, "fp32")
    for x, y, sp in zip(xs, ys, specs):
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, 1e-3)
        p = fbf.make_params(c, sp["sigma_s"], sp.get("W", 0), sp.get("spatial", "gaussian"), "reflect", per_form)
        single = fbf.fbf_filter(p, x)
        torch.cuda.synchronize()
        if kind.startswith("per_image"):
            assert torch.equal(single, y)
        else:  # box windows: FIR in the persistent kernels, running sums in the single-image one
            tol = 2e-3 if sp.get("spatial") == "box" else 1e-4
            assert torch.max(torch.abs(single - y)).item() <= tol
    plan.destroy()


FORM_SCHEDULES = {
    "fp32": ["persistent", "persistent_wide", "per_image_fp32", "per_image_fp32_streams"],
    "auto": ["persistent", "persistent_wide", "per_image_fp32", "per_image_fp32_streams", "per_image_form",
             "per_image_form_streams"],
    "tc_fp16_single": ["per_image_form", "per_image_form_streams", "persistent_tc"],
}


@pytest.mark.parametrize("form,schedule", [(f, k) for f, ks in FORM_SCHEDULES.items() for k in ks])
def test_every_schedule_explicitly(fbf, form, schedule):
    """Each candidate schedule captured on its own (fbf_plan_create_schedule):
    per-image schedules, sequential or on concurrent branches, replay exactly
    the single-image kernels (bit-identical); the persistent ones the FP32 tile
    body with run-time taps (within 1e-4).  Two replays give the same result."""
    import torch

    shapes = [(300, 260), (70, 90), (33, 200), (256, 40), (130, 131), (1, 64), (200, 180), (90, 300)]
    specs = [dict(sigma_s=3.0, sigma_r=30.0), dict(sigma_s=0.7, sigma_r=15.0), dict(sigma_s=5.0, sigma_r=50.0),
             dict(sigma_s=2.0, sigma_r=60.0, eps=1e-2), dict(sigma_s=4.0, sigma_r=25.0), dict(sigma_s=1.5, sigma_r=20.0),
             dict(sigma_s=2.5, sigma_r=40.0), dict(sigma_s=1.0, sigma_r=35.0)]
    imgs = [make_image(h, w, seed=1600 + k) for k, (h, w) in enumerate(shapes)]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    ys = [torch.full(im.shape, float("nan"), dtype=torch.float32, device="cuda") for im in imgs]
    plan = fbf.fbf_plan_create(xs, ys, specs, form, "reflect", schedule=schedule)
    assert plan.schedule() == (schedule, 0.0)
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    first = [y.clone() for y in ys]
    for y in ys:
        y.fill_(float("nan"))
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    per_form = "fp32" if schedule in ("per_image_fp32", "per_image_fp32_streams", "persistent", "persistent_wide") \
        else form
    for x, y, y0, sp in zip(xs, ys, first, specs):
        assert torch.equal(y, y0)
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, sp.get("eps", 1e-3))
        p = fbf.make_params(c, sp["sigma_s"], 0, "gaussian", "reflect", per_form)
        single = fbf.fbf_filter(p, x)
        torch.cuda.synchronize()
        if schedule.startswith("per_image") or schedule == "persistent_tc":
            assert torch.equal(single, y)  # the same tile arithmetic as the single-image kernels
        else:
            assert torch.max(torch.abs(single - y)).item() <= 1e-4
    plan.destroy()


def test_schedule_not_of_the_form_is_rejected(fbf):
    import ctypes as C

    import torch

    x = torch.zeros((40, 40), dtype=torch.uint8, device="cuda")
    y = torch.zeros((40, 40), dtype=torch.float32, device="cuda")
    for form, schedule in (("tc_fp16", "persistent"), ("tc_fp16", "per_image_fp32_streams"),
                           ("fp32", "per_image_form"), ("fp32", "persistent_tc"), ("tc_fp16", "persistent_tc"),
                           ("auto", "persistent_tc")):
        with pytest.raises(fbf.FbfError) as e:
            fbf.fbf_plan_create([x], [y], [dict(sigma_s=2.0, sigma_r=30.0)], form, schedule=schedule)
        assert e.value.status == fbf.FBF_ERR_INVALID_ARGUMENT
    h = C.c_void_p()
    arr = (fbf.fbf_image_desc * 1)()
    assert fbf.lib.fbf_plan_create_schedule(arr, 0, fbf.FBF_FORM_FP32, 0, 6, C.byref(h)) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert fbf.lib.fbf_plan_create_schedule(arr, 0, fbf.FBF_FORM_TC_FP16_SINGLE, 0, 7, C.byref(h)) == \
        fbf.FBF_ERR_INVALID_ARGUMENT
    assert fbf.lib.fbf_plan_create_schedule(arr, 0, fbf.FBF_FORM_FP32, 0, -1, C.byref(h)) == \
        fbf.FBF_ERR_INVALID_ARGUMENT


@pytest.mark.parametrize("form", ["tc_fp16", "tc_fp16_single", "tc_bf16"])
def test_tensor_core_plan(fbf, form):
    """Tensor-core plans replay one launch per image (on one or on concurrent
    graph branches): identical to fbf_filter in that form, and within the
    form's tolerance of the oracle."""
    import torch

    shapes = [(70, 90), (33, 200), (256, 40), (130, 131), (300, 260)]
    specs = [dict(sigma_s=3.0, sigma_r=30.0), dict(sigma_s=0.7, sigma_r=15.0), dict(sigma_s=6.0, sigma_r=50.0),
             dict(sigma_s=2.0, sigma_r=60.0, eps=1e-2), dict(sigma_s=10.0, sigma_r=25.0)]
    imgs = [make_image(h, w, seed=1500 + k) for k, (h, w) in enumerate(shapes)]
    plan, xs, ys = _run_plan(fbf, imgs, specs, form=form)
    kinds = ("per_image_form", "per_image_form_streams") + (("persistent_tc",) if form == "tc_fp16_single" else ())
    assert plan.schedule()[0] in kinds
    tol = 0.15 if form == "tc_fp16_single" else 0.02
    for im, x, y, sp in zip(imgs, xs, ys, specs):
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, sp.get("eps", 1e-3))
        p = fbf.make_params(c, sp["sigma_s"], 0, "gaussian", "reflect", form)
        single = fbf.fbf_filter(p, x)
        torch.cuda.synchronize()
        assert torch.equal(single, y)
        W = int(np.ceil(3 * sp["sigma_s"] - 1e-12))
        ref = O.alg1(im, O.weights_1d(O.SPATIAL_GAUSSIAN, sp["sigma_s"], W), O.BORDER_REFLECT,
                     np.array(c.coefficients), 255.0)[0]
        assert np.abs(y.cpu().numpy() - ref).max() <= tol
    plan.destroy()


# Per window band of the persistent tensor-core kernel (its instantiation follows
# the batch's largest W: 16, 32, 48), the (sigma_s, sigma_r) of eight images.
PTC_SPECS = {
    16: [(3.0, 30.0), (0.7, 15.0), (5.0, 50.0), (2.0, 60.0), (4.0, 15.0), (1.5, 20.0), (5.3, 40.0), (1.0, 35.0)],
    32: [(3.0, 30.0), (10.0, 20.0), (6.0, 50.0), (2.0, 60.0), (8.3, 25.0), (1.5, 20.0), (10.6, 40.0), (7.0, 15.0)],
    48: [(16.0, 30.0), (3.0, 20.0), (12.0, 50.0), (11.0, 60.0), (14.2, 25.0), (1.5, 20.0), (6.0, 40.0), (15.9, 15.0)],
}


@pytest.mark.parametrize("border", ["reflect", "truncate"])
@pytest.mark.parametrize("band", [16, 32, 48])
def test_persistent_tc_plan_matches_oracle(fbf, band, border):
    """The persistent tensor-core schedule (one launch over cost-sorted (image,
    tile) items of all images; Algorithm 1 per image with its own K from
    Algorithm 2): ragged shapes down to 1 x 64 and 5 x 7, one image read through a
    strided view whose pitch breaks TMA's 16-byte rule (plain loads), windows
    of every band.  Every output equals the single-image filter of the same form
    bit for bit and Algorithm 1 in FP64 within the form's tolerance; a second
    replay gives the same outputs."""
    import torch

    shapes = [(300, 260), (70, 90), (33, 200), (256, 40), (1, 64), (5, 7), (130, 131), (129, 97)]
    imgs = [make_image(h, w, seed=1700 + 10 * band + k) for k, (h, w) in enumerate(shapes)]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    big = torch.zeros((140, 141), dtype=torch.uint8, device="cuda")  # pitch 141: no TMA map
    big[3:3 + 129, 5:5 + 97] = xs[7]
    xs[7] = big[3:3 + 129, 5:5 + 97]
    ys = [torch.full(im.shape, float("nan"), dtype=torch.float32, device="cuda") for im in imgs]
    specs = [dict(sigma_s=ss, sigma_r=sr) for ss, sr in PTC_SPECS[band]]
    assert max(int(np.ceil(3 * s["sigma_s"] - 1e-12)) for s in specs) > band - 16
    plan = fbf.fbf_plan_create(xs, ys, specs, "tc_fp16_single", border, schedule="persistent_tc")
    assert plan.schedule() == ("persistent_tc", 0.0)
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    first = [y.clone() for y in ys]
    for y in ys:
        y.fill_(float("nan"))
    fbf.fbf_filter_batched(plan)
    torch.cuda.synchronize()
    bd = O.BORDER_REFLECT if border == "reflect" else O.BORDER_TRUNCATE
    for im, x, y, y0, sp in zip(imgs, xs, ys, first, specs):
        assert torch.equal(y, y0)
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, 1e-3)
        p = fbf.make_params(c, sp["sigma_s"], 0, "gaussian", border, "tc_fp16_single")
        single = fbf.fbf_filter(p, x)
        torch.cuda.synchronize()
        assert torch.equal(single, y)
        W = int(np.ceil(3 * sp["sigma_s"] - 1e-12))
        ref = O.alg1(im, O.weights_1d(O.SPATIAL_GAUSSIAN, sp["sigma_s"], W), bd, np.array(c.coefficients), 255.0)[0]
        assert np.abs(y.cpu().numpy() - ref).max() <= 0.15
    plan.destroy()


def test_persistent_tc_plan_is_autotuned_on_an_uneven_batch(fbf):
    """Form TC_FP16_SINGLE on a 32-image uneven batch: the autotuner times the
    persistent tensor-core launch against the per-image schedules; whichever it
    keeps, every output equals the single-image filter."""
    import torch

    specs_raw = make_batch_specs(32, seed=1399, lo=64, hi=600)
    imgs = [make_image(h, w, seed=s) for (h, w, _, _, s) in specs_raw]
    specs = [dict(sigma_s=ss, sigma_r=sr) for (_, _, ss, sr, _) in specs_raw]
    plan, xs, ys = _run_plan(fbf, imgs, specs, form="tc_fp16_single")
    kind, ms = plan.schedule()
    assert kind in ("persistent_tc", "per_image_form", "per_image_form_streams") and ms > 0
    for x, y, sp in zip(xs, ys, specs):
        c = fbf.fbf_fit_coeffs("gaussian", sp["sigma_r"], 255.0, 1e-3)
        single = fbf.fbf_filter(fbf.make_params(c, sp["sigma_s"], 0, "gaussian", "reflect", "tc_fp16_single"), x)
        torch.cuda.synchronize()
        assert torch.equal(single, y)
    plan.destroy()


def test_tuning_cache_reuses_the_autotuned_schedule(fbf, tmp_path):
    """With a tuning cache the first plan autotunes and records its choice; a
    second plan for the same request on this GPU captures that schedule without
    replaying the candidates (autotune time 0) and gives the same outputs."""
    import json

    import torch

    path = str(tmp_path / "tune.json")
    specs_raw = make_batch_specs(12, seed=1399, lo=64, hi=400)
    imgs = [make_image(h, w, seed=s) for (h, w, _, _, s) in specs_raw]
    specs = [dict(sigma_s=ss, sigma_r=sr) for (_, _, ss, sr, _) in specs_raw]
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    ys = [torch.empty(im.shape, dtype=torch.float32, device="cuda") for im in imgs]
    p1 = fbf.fbf_plan_create(xs, ys, specs, "tc_fp16_single", "reflect", tune_cache=path)
    kind, ms = p1.schedule()
    assert ms > 0
    entries = json.load(open(path))["entries"][torch.cuda.get_device_name()]
    assert [e["schedule"] for e in entries.values()] == [kind]
    fbf.fbf_filter_batched(p1)
    torch.cuda.synchronize()
    first = [y.clone() for y in ys]
    p2 = fbf.fbf_plan_create(xs, ys, specs, "tc_fp16_single", "reflect", tune_cache=path)
    assert p2.schedule() == (kind, 0.0)
    for y in ys:
        y.fill_(float("nan"))
    fbf.fbf_filter_batched(p2)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(first, ys))
    p1.destroy()
    p2.destroy()
