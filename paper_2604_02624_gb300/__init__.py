"""GB300-native forward model and adjoint of wavelength-multiplexed diffractive storage."""
