"""Frozen-flow layers on infinite phase screens (AtmoInfiniteEvolution, Tab. 4;
InfinitePhaseScreen, Tab. 3).

Each layer keeps a side x side ring screen.  Column line L sits at column
L mod side and row line L at row L mod side, and the layer extraction's
periodic addressing reads the ring unchanged.  Before each frame, the rows
and columns the layer's footprint needs at time t are grown by
``specula_infscreen_lines``.  Each new line is a Gaussian draw conditioned on
the lines behind it, with the noise keyed by (seed, layer, axis, line).  A
screen's content therefore depends only on how far it has moved, not on the
frame timing.  The rings start as FFT screens of the same side.

This class owns the rings, the operators and the window state; the library
plans each frame's lines (``specula_infscreen_advance``, native) and grows
them in its kernels.
"""
import ctypes as C

import synth
from . import (INF_MAX_TASKS, LayerDesc, _abi, _stream, layer_desc, lib, pupil_desc,
               source_desc, specula_infscreen_operators, specula_screen_generate)


class InfiniteAtmosphere:
    def __init__(self, ctx, layers, source, pupil, side, n_st=2, seed=1, rcond=1e-12,
                 device="cuda", margin=1):
        """layers: synth Layer records (pitch_m, height_m, vx_mps, vy_mps, r0_m,
        L0_m, seed; their `side` is replaced by the ring's); source, pupil: synth
        Source and Pupil records of the extraction that reads the rings."""
        import torch
        self.ctx, self.side, self.n_st, self.seed = ctx, int(side), int(n_st), int(seed)
        self.layers, self.src, self.pupil, self.margin = list(layers), source, pupil, int(margin)
        if len(self.layers) > INF_MAX_TASKS:
            raise ValueError(f"at most {INF_MAX_TASKS} infinite layers")
        self.ops = {}
        for l in self.layers:
            key = (float(l.pitch_m), float(l.L0_m))
            if key not in self.ops:
                r0_ref = float(l.r0_m)
                A, B = specula_infscreen_operators(ctx, self.side, self.n_st, l.pitch_m, r0_ref,
                                                   l.L0_m, rcond)
                self.ops[key] = (A, B, r0_ref)
        self.screens = []
        for l in self.layers:
            noise = torch.tensor(synth.screen_noise(l.seed, self.side), device=device)
            scr = torch.empty(self.side, self.side, device=device, dtype=torch.float32)
            specula_screen_generate(ctx, self.side, l.pitch_m, l.r0_m, l.L0_m, noise,
                                    synth.subharmonic_noise(l.seed), scr)
            self.screens.append(scr)
        # window state: lowest line per (layer, axis 0 rows / 1 columns); the
        # FFT screen holds lines 0 .. side-1
        n = len(self.layers)
        descs = []
        for l in self.layers:
            d = layer_desc(l)
            d.side = self.side
            descs.append(d)
        self._layers = (LayerDesc * n)(*descs)
        self._src = source_desc(source)
        self._pupil = pupil_desc(pupil)
        self._lo = (C.c_int64 * (2 * n))()
        self._scr = (C.c_void_p * n)(*[x.data_ptr() for x in self.screens])
        keys = [(float(l.pitch_m), float(l.L0_m)) for l in self.layers]
        self._A = (C.c_void_p * n)(*[self.ops[k][0].data_ptr() for k in keys])
        self._B = (C.c_void_p * n)(*[self.ops[k][1].data_ptr() for k in keys])
        self._bs = (C.c_float * n)(*[(self.ops[k][2] / float(l.r0_m)) ** (5.0 / 6.0)
                                     for k, l in zip(keys, self.layers)])
        self.lines_grown = 0
        self.advance(0.0)          # checks that every footprint fits its ring

    @property
    def lo(self):
        """Per layer [rows, columns] lowest line of the ring window."""
        return [[self._lo[2 * i], self._lo[2 * i + 1]] for i in range(len(self.layers))]

    def advance(self, t, stream=None):
        """Grow every layer's ring to cover its footprint at time t (native
        plan, then one kernel per round of lines); returns the number of
        kernel calls."""
        n = len(self.layers)
        calls = C.c_int32()
        lo0 = list(self._lo)
        _abi.check(lib().specula_infscreen_advance(
            self.ctx.handle, n, C.cast(self._layers, C.c_void_p), C.byref(self._src),
            C.byref(self._pupil), self.side, self.n_st, self.margin,
            C.cast(self._scr, C.c_void_p), C.cast(self._A, C.c_void_p),
            C.cast(self._B, C.c_void_p), C.cast(self._bs, C.c_void_p),
            C.cast(self._lo, C.c_void_p), float(t), C.c_uint64(self.seed), C.byref(calls),
            _stream(stream)), "specula_infscreen_advance")
        self.lines_grown += sum(abs(a - b) for a, b in zip(self._lo, lo0))
        return calls.value
