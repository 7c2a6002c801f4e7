"""GB300-native wave-based NLOS reconstruction (confocal f-k migration and
phasor-field RSD) behind a small C ABI.

The compute path lives in the CUDA library built from `csrc/`; `nlos` is its
thin Python binding (argument marshalling only). `synth` renders seeded
synthetic captures.
"""
__all__ = ["nlos", "synth"]
