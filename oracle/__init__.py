"""FP64 CPU oracle of the wavefront-sensor forward model.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
it may be used by ``tests/``, by ``__graft_entry__.smoke()`` (to check one
small GPU invocation) and by ``bench.py``'s CPU-baseline / reference legs.  It
shares no code, table or constant generator with the CUDA library; the only
code both sides use is the seeded input generator package ``synth``.

The paper (a framework paper) names the processing objects of the hot path
(App. A, Tab. 4: AtmoEvolution, AtmoPropagation, ModulatedPyramid, SH, CCD,
PyrSlopec, ShSlopec, Modalrec, ImCalibrator, RecCalibrator) and their
parameters (App. B, Listing 2) but prints no equation for them.  This oracle
writes the textbook physics of those objects out in plain NumPy, in float64,
with ``numpy.fft`` (pocketfft) as the only library primitive for the
transforms.  Every reading of a point the paper leaves open is stated in the
docstring of the function that makes it.

Modules and their pins (tests/test_oracle_*.py):

* ``dft``       centred DFT; pinned to a brute-force O(n^4) sum.
* ``geometry``  pupil stop, valid subapertures, quadrant index maps,
                modulation angles; pinned to hand-counted tiny cases and to
                symmetry counts.
* ``screens``   von Karman FFT screens with subharmonics; pinned to the exact
                ensemble structure function, the Kolmogorov 5/3 law and the
                phase variance.
* ``atmo``      frozen-flow layer extraction; pinned to exact rolls, linear
                ramps (bilinear reproduces them) and the zero-height on-axis
                identity.
* ``pyramid``   modulated pyramid intensity and binning; pinned to Parseval
                flux, mirror/transpose symmetries, equal quadrant flux, tilt
                antisymmetry, and the unit-mask identity.  Its shifted-mask
                form is pinned to the tilt form for whole-bin shifts of a
                band-limited field and without modulation, to a brute-force
                tiny case, Parseval flux and the flat-wavefront symmetries.
* ``sh``        Shack-Hartmann spots; pinned to zero centroid for a flat
                wavefront, exact circular roll under an integer tilt, and
                per-subaperture Parseval flux.
* ``pyramid.rebin_area``  area-weighted detector rebinning for a
                non-integer pixel ratio; pinned to exact rational interval
                overlaps, block binning at integer ratios, flux, a constant
                image and a hand-placed point source.
* ``slopes``    pyramid and centre-of-gravity slopes; pinned through the
                pyramid / SH invariants above and hand-computed detectors.
* ``recon``     modal reconstructor MVM; pinned to a direct sum.
* ``modal``     Zernike modal basis (Noll order) and least-squares projection;
                pinned to the Noll table, closed forms of low orders,
                continuous orthonormality and exact coefficient recovery.
* ``calib``     push-pull interaction matrix and truncated pseudo-inverse;
                pinned to the Penrose conditions, tip/tilt transpose symmetry
                and sign, and reconstructor closure R IM = I on kept modes.
* ``mlp``       learned reconstructor (GELU perceptron, MSE, Adam); pinned to
                erf values of GELU, central finite differences of the
                backward pass, the first Adam step and a training decrease.
* ``philox``    Philox4x32-10 counter-based generator and Box-Muller normals;
                pinned to the published known-answer vectors.
* ``system``    a multi-sensor system: the chains above per sensor, slopes
                concatenated; pinned to zero slopes for flat screens, equal
                SH slopes in every subaperture for a linear phase ramp, and
                block-wise agreement with the single-sensor chains.
* ``ccd``       detector photon (Poisson) and readout noise from Philox draws;
                pinned to the Poisson mean, variance and zero-count
                probability in both samplers, the readout normal's moments
                and determinism per (seed, frame).
* ``loop``      the closed loop (modal mirror, integrator, one-step delay)
                and its residual RMS / Strehl ratio; pinned to the scalar
                recursion of an ideal sensor on a static modal aberration,
                the zero-gain identity and closed-form statistics.
* ``infinite``  infinite phase screens grown line by line from the Gaussian
                conditional on a stencil of lines; pinned to a numerical
                Hankel transform of the screens' spectrum, the variance
                integral, the small-separation Bessel expansion, the joint
                covariance and the precision-matrix form of the conditional,
                exact mirror / transpose identities, and the structure
                function of a long grown strip.
"""
